// vq_resident_rc2.cu -- resident-kernel variants with 2 replica(s) per CTA.
#include "vq_resident_kernel.cuh"

namespace vq {

resident::KFn resident_pick_rc2(int rpt, bool csr_smem, bool packed, bool ell) {
    return resident::pick_rpt<2>(rpt, csr_smem, packed, ell);
}

}  // namespace vq
