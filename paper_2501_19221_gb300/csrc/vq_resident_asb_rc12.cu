// vq_resident_asb_rc12.cu -- resident-kernel variants of the adiabatic-SB form
// with 1 or 2 replicas per CTA.
#include "vq_resident_kernel.cuh"

namespace vq {

VQ_RESIDENT_PICK(1, 1) { return resident::pick_rpt<1, 1>(rpt, csr_smem, packed, ell, threads); }
VQ_RESIDENT_PICK(2, 1) { return resident::pick_rpt<2, 1>(rpt, csr_smem, packed, ell, threads); }

}  // namespace vq
