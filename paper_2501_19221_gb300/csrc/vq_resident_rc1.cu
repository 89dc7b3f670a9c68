// vq_resident_rc1.cu -- resident-kernel variants with 1 replica(s) per CTA.
#include "vq_resident_kernel.cuh"

namespace vq {

resident::KFn resident_pick_rc1(int rpt, bool csr_smem, bool packed, bool ell) {
    return resident::pick_rpt<1>(rpt, csr_smem, packed, ell);
}

}  // namespace vq
