// pond_adjoint.cu -- vector-Jacobian product of one PonD step (placeholder
// until the adjoint kernels land).
#include "pond_device.cuh"

namespace pond {

__constant__ Lattice c_La;

cudaError_t upload_lattice_adjoint(const Lattice& L) {
    return cudaMemcpyToSymbol(c_La, &L, sizeof(Lattice));
}

}  // namespace pond

void destroy_adjoint(pond_ctx*) {}

extern "C" pond_status pond_adjoint_step(pond_ctx* ctx, const void*, const void*, void*, void*,
                                         double*) {
    if (!ctx) return POND_ERR_ARG;
    ctx->err = "adjoint not available in this build";
    return POND_ERR_STATE;
}
