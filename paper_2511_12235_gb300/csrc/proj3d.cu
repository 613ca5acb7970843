// proj3d.cu -- 3D cone-beam projectors (placeholder until the 3D kernels land).
#include "csm_internal.cuh"

namespace csm {

size_t workspace_3d(const csm_geom_s*, int, int64_t, bool) { return 0; }

csm_status forward_3d(const csm_geom_s*, const void*, void*, int64_t, csm_dtype, csm_dtype, int, void*, size_t,
                      cudaStream_t) {
    return CSM_EUNSUPPORTED;
}

csm_status back_3d(const csm_geom_s*, const void*, void*, int64_t, csm_dtype, csm_dtype, int, void*, size_t,
                   cudaStream_t) {
    return CSM_EUNSUPPORTED;
}

csm_status nnz_3d(const csm_geom_s*, int64_t*, cudaStream_t) { return CSM_EUNSUPPORTED; }

}  // namespace csm
