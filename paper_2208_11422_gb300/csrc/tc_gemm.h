// Tensor-core (tcgen05) implicit-GEMM projections: interface used by lfd_api.cu.
#pragma once
#include "lfd_internal.h"

namespace lfd {

// number of partial outputs the forward / backward kernels write for a shape
int tc_forward_parts_for(const Geo& g, int sm_count);
int tc_backward_parts_for(const Geo& g, int sm_count);
int tc_forward_parts(const lfd_ctx* ctx);
int tc_backward_parts(const lfd_ctx* ctx);

// builds the TMA tensor maps and launch plans (once per context)
cudaError_t tc_init(lfd_ctx* ctx);
// Hv partials of the BF16 copies of Vp32[buf] into ctx->Fwd
cudaError_t tc_forward(lfd_ctx* ctx, int buf, cudaStream_t st);
// H^T r partials of the BF16 copies of Rp32 into ctx->Bwd
cudaError_t tc_backward(lfd_ctx* ctx, cudaStream_t st);
void tc_destroy(lfd_ctx* ctx);
// shape check: the forward tile holds all Nnum^2 phases (<= 256 columns)
bool tc_supported(const Geo& g);
// error word of the tensor-core kernels (0 = none; 1-4 = which wait timed
// out); reading it synchronises with the device and clears it
int tc_error(lfd_ctx* ctx);

}  // namespace lfd
