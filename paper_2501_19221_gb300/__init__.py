"""GB300 (sm_103a) implementation of the data-parallel hot path of the VeloxQ
QUBO solver (arXiv:2501.19221): replicas of a ballistic simulated-bifurcation
system integrated in lockstep, with the local field, fused update/readout and
exact energies in hand-written CUDA behind a C ABI (include/veloxq.h).

``binding`` is the ctypes binding of that ABI; ``instances`` the seeded
synthetic instance generators; ``replicas`` the post-run exchanges of
replica parallelism over several processes. Importing ``binding`` needs the compiled
library (``__graft_entry__.build()``).
"""
__all__ = ["binding", "instances", "replicas"]
