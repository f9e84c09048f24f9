// Discrete adjoint entry points (implementation in progress in this file).
#include "../../include/alsv.h"

extern "C" {
alsv_status alsv_adjoint_workspace_bytes(alsv_ctx*, double, size_t* bytes) {
    if (bytes) *bytes = 0;
    return ALSV_ERR_INVALID_ARG;
}
alsv_status alsv_bind_adjoint_workspace(alsv_ctx*, void*, size_t) { return ALSV_ERR_INVALID_ARG; }
alsv_status alsv_adjoint_evolve(alsv_ctx*, double, int, const double*, double*, double*) { return ALSV_ERR_INVALID_ARG; }
}
