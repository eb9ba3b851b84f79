// Adjoint kernels (bin-mode DOS backward, eigensolver backward).
#include "tetra_internal.cuh"

namespace tetra {

size_t dos_backward_workspace(const Plan &P) { return kStatusBytes; }

tetra_status_t launch_dos_backward(const Plan &, const float *, const void *, const float *,
                                   const float *, float *, float *, void *, size_t, cudaStream_t) {
    return TETRA_EUNSUPPORTED;
}

size_t eig_backward_workspace(const Plan &P, int n_R) { return kStatusBytes; }

tetra_status_t launch_eig_backward(const Plan &, const tetra_model_t *, const float *,
                                   const float *, float *, void *, size_t, cudaStream_t) {
    return TETRA_EUNSUPPORTED;
}

}  // namespace tetra
