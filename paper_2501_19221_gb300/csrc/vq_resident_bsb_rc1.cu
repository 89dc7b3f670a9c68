// vq_resident_bsb_rc1.cu -- resident-kernel variants of the ballistic form with 1
// replica(s) per CTA.
#include "vq_resident_kernel.cuh"

namespace vq {

VQ_RESIDENT_PICK(1, 0) { return resident::pick_rpt<1, 0>(rpt, csr_smem, packed, ell, threads); }

}  // namespace vq
