// vq_resident_pa_rc12.cu -- resident-kernel variants of the Parallel-Annealing form
// with 1 or 2 replicas per CTA.
#include "vq_resident_kernel.cuh"

namespace vq {

VQ_RESIDENT_PICK(1, 2) { return resident::pick_rpt<1, 2>(rpt, csr_smem, packed, ell, threads); }
VQ_RESIDENT_PICK(2, 2) { return resident::pick_rpt<2, 2>(rpt, csr_smem, packed, ell, threads); }

}  // namespace vq
