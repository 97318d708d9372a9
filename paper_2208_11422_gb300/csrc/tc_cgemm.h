// Split-BF16 complex contractions of the FFT variant on tcgen05 (tc_cgemm.cu).
#pragma once
#include <string>

#include "lfd_internal.h"

namespace lfd {

// Operands are BF16 planes: [0] real hi, [1] real lo, [2] imag hi, [3] imag lo.
struct CgemmBuffers {
    int bins, ntile;          // frequency bins; tiles per frame
    int ncolp;                // columns of the X / Y planes (padded to 16)
    int S, C;                 // phases, channels
    int Sw, Cw;               // plane row lengths (multiples of 8)
    int Sf, Cf;               // FP32 complex output row lengths
    const __nv_bfloat16* W[4];  // [bins][S][Cw] PSF spectra
    const __nv_bfloat16* X[4];  // [Cw/8][ncolp][bins][8] volume spectra (forward input)
    const __nv_bfloat16* Y[4];  // [Sw/8][ncolp][bins][8] ratio spectra (adjoint input)
    float2* Yout;             // [bins][ncol][Sf] forward output
    float2* Xout;             // [bins][ncol][Cf] adjoint output
};

cudaError_t cgemm_init(const CgemmBuffers& b, int sm_count, void** state, std::string* why);
// ncol = frames x tiles of this call (<= ncolp)
cudaError_t cgemm_forward(void* state, int ncol, cudaStream_t st);
cudaError_t cgemm_adjoint(void* state, int ncol, cudaStream_t st);
int cgemm_error(void* state);  // 0, or the code of a wait that gave up (11-14)
void cgemm_destroy(void* state);

}  // namespace lfd
