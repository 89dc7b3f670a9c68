// vq_resident_rc4.cu -- resident-kernel variants with 4 replica(s) per CTA.
#include "vq_resident_kernel.cuh"

namespace vq {

resident::KFn resident_pick_rc4(int rpt, bool csr_smem, bool packed, bool ell) {
    return resident::pick_rpt<4>(rpt, csr_smem, packed, ell);
}

}  // namespace vq
