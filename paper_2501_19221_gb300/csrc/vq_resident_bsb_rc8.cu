// vq_resident_bsb_rc8.cu -- resident-kernel variants of the ballistic form with 8
// replica(s) per CTA.
#include "vq_resident_kernel.cuh"

namespace vq {

VQ_RESIDENT_PICK(8, 0) { return resident::pick_rpt<8, 0>(rpt, csr_smem, packed, ell, threads); }

}  // namespace vq
