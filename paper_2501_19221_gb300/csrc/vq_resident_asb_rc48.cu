// vq_resident_asb_rc48.cu -- resident-kernel variants of the adiabatic-SB form
// with 4 or 8 replicas per CTA.
#include "vq_resident_kernel.cuh"

namespace vq {

VQ_RESIDENT_PICK(4, 1) { return resident::pick_rpt<4, 1>(rpt, csr_smem, packed, ell, threads); }
VQ_RESIDENT_PICK(8, 1) { return resident::pick_rpt<8, 1>(rpt, csr_smem, packed, ell, threads); }

}  // namespace vq
