// Split-BF16 complex contractions of the FFT variant on tcgen05 (tc_cgemm.cu).
#pragma once
#include <string>
#include <vector>

#include "lfd_internal.h"

namespace lfd {

// Adaptive lo planes of the PSF spectra (cgemm_compact_lo): the lo planes of
// the (bin, 64-channel block) tiles whose largest hi value reaches tau x the
// largest of all, as compact planes [kept + 1][S][64] (slot 0 all zeros), and
// slot[bin][block] (0: dropped).
struct LoPlanes {
    __nv_bfloat16* lo[2] = {};  // real lo, imag lo
    int* slot = nullptr;
    int nkbc = 0;               // 64-channel blocks per bin
    int64_t kept = 0, tiles = 0;
};

// The forward's copy of the adaptive PSF spectra in the order its wide units
// read them (cgemm_build_wide): per bin and k-block of 16 channels, for row
// tile m (rows [128 m, 128 m + rows_m) of the S phases), plane (real, imag)
// and channel group g (8 channels), the rows_m x 16 bytes of the canonical
// K-major core-matrix layout [g][row][8], valid rows only:
//   hi[bin][kb16][m][plane][g][rows_m][8]   (64 S bytes per bin and k-block)
//   lo[slot][kb16 % 4][m][plane][g][rows_m][8] for the slots of LoPlanes
// (a 64-channel block is four k-blocks). One unit of the wide forward kernel
// covers both bins of a 32-byte sector of the data planes and both row tiles.
struct WidePlanes {
    __nv_bfloat16* hi = nullptr;
    __nv_bfloat16* lo = nullptr;
    int nkb16 = 0;              // k-blocks of 16 channels per bin
};

// Operands are BF16 planes: [0] real hi, [1] real lo, [2] imag hi, [3] imag lo.
// The PSF spectra: all four planes (split BF16), the two hi planes (W[1], W[3]
// null: BF16 spectra), or the two hi planes and lo.slot != null (adaptive).
struct CgemmBuffers {
    int bins, ntile;          // frequency bins; tiles per frame
    int ncolp;                // columns of the X / Y planes (padded to 16)
    int S, C;                 // phases, channels
    int Sw, Cw;               // plane row lengths (multiples of 8)
    int Sf, Cf;               // FP32 complex output row lengths
    const __nv_bfloat16* W[4];  // [bins][S][Cw] PSF spectra
    const __nv_bfloat16* X;   // [Cw/8][4 planes][ncolp][bins][8] volume spectra (forward input)
    const __nv_bfloat16* Y;   // [Sw/8][4 planes][ncolp][bins][8] ratio spectra (adjoint input)
    float2* Yout;             // [Sf/8][ncol][bins][8] forward output (group-major)
    float2* Xout;             // [Cf/8][bins][ncol][8] adjoint output (group-major, columns inner)
    LoPlanes lo;              // adaptive lo planes (slot null otherwise)
    int max_cols;             // widest column chunk (16, 32 or 64); 0: up to 64
    WidePlanes wide;          // the forward's wide-unit copy (hi null: not used)
};

// Builds the adaptive lo planes from the full planes b.W[0..3] ([bins][S][Cw]);
// the caller may free b.W[1] and b.W[3] afterwards. Device bytes allocated
// are added to *bytes.
cudaError_t cgemm_compact_lo(const CgemmBuffers& b, float tau, cudaStream_t st, LoPlanes* out, int64_t* bytes);
void cgemm_free_lo(LoPlanes* p);

// Builds the wide-unit copy of the adaptive spectra from the hi planes b.W[0],
// b.W[2] ([bins][S][Cw]) and the compact lo planes `lo`; S <= 256. Device
// bytes allocated are added to *bytes.
cudaError_t cgemm_build_wide(const CgemmBuffers& b, const LoPlanes& lo, cudaStream_t st, WidePlanes* out,
                             int64_t* bytes);
void cgemm_free_wide(WidePlanes* p);

// contiguous ranges of about equal total cost over units 0 .. cost.size()-1
// for `grid` blocks: block k takes units [st[k], st[k+1]) (tc_cgemm.cu)
std::vector<int64_t> balanced_ranges(const std::vector<double>& cost, int grid);

cudaError_t cgemm_init(const CgemmBuffers& b, int sm_count, void** state, std::string* why);
// ncol = frames x tiles of this call (<= ncolp)
cudaError_t cgemm_forward(void* state, int ncol, cudaStream_t st);
cudaError_t cgemm_adjoint(void* state, int ncol, cudaStream_t st);
int cgemm_error(void* state);  // 0, or the code of a wait that gave up (11-16)
void cgemm_destroy(void* state);

}  // namespace lfd
