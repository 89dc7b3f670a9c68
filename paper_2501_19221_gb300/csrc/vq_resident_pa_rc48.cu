// vq_resident_pa_rc48.cu -- resident-kernel variants of the Parallel-Annealing form
// with 4 or 8 replicas per CTA.
#include "vq_resident_kernel.cuh"

namespace vq {

VQ_RESIDENT_PICK(4, 2) { return resident::pick_rpt<4, 2>(rpt, csr_smem, packed, ell, threads); }
VQ_RESIDENT_PICK(8, 2) { return resident::pick_rpt<8, 2>(rpt, csr_smem, packed, ell, threads); }

}  // namespace vq
