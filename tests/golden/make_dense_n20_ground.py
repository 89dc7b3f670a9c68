"""Write dense_n20_ground.txt: the ground energy of the dense n = 20 integer
QUBO (entries uniform in [-8, 8], symmetric, seed 0) and the number of
minimisers, by exhaustive enumeration of all 2^20 assignments in the oracle.

    python tests/golden/make_dense_n20_ground.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_2501_19221_gb300 import instances as I  # noqa: E402


def main():
    Q, c = I.dense_int_qubo(20, seed=0)
    E, x, count = O.bruteforce(O.problem_from_dense(Q, c))
    with open(os.path.join(HERE, "dense_n20_ground.txt"), "w") as f:
        f.write("# dense n=20 integer QUBO, entries uniform in [-8, 8], symmetric, seed 0;\n")
        f.write("# exhaustive enumeration of 2^20 assignments by the oracle (make_dense_n20_ground.py)\n")
        f.write(f"E_min {int(E)}\n")
        f.write(f"minimisers {int(count)}\n")
        f.write("x_min " + "".join(str(int(v)) for v in x) + "\n")


if __name__ == "__main__":
    main()
