// vq_resident_rc8.cu -- resident-kernel variants with 8 replica(s) per CTA.
#include "vq_resident_kernel.cuh"

namespace vq {

resident::KFn resident_pick_rc8(int rpt, bool csr_smem, bool packed, bool ell) {
    return resident::pick_rpt<8>(rpt, csr_smem, packed, ell);
}

}  // namespace vq
