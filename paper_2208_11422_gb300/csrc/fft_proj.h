// FFT (overlap-save) variant of the projections: interface used by lfd_api.cu.
#pragma once
#include "lfd_internal.h"

namespace lfd {

struct FftPlan {
    int F = 0;          // transform size per axis (32 or 64)
    int B = 0;          // valid outputs per tile and axis, F - 2h
    int h = 0;          // tap halo
    int tiles_y = 0, tiles_x = 0, ntile = 0;
    int bins = 0;       // F * (F/2 + 1)
    int Cf = 0, Sf = 0; // channel / phase counts padded to 8 (row lengths of the complex64
                        // spectra; the inverse transform reads whole 8-channel groups)
    int Cw = 0, Sw = 0; // padded to 8 (row lengths of the BF16 planes)
};

// Spectra buffers. FP32 contraction: Wf, Xh, Yh (complex64). Tensor-core
// contraction (cg != null): BF16 planes (real hi, real lo, imag hi, imag lo)
// Wp[4] [bins][S][Cw] (PSF); the volume and ratio columns in one block each,
// [Cw/8][4 planes][ncolp][bins][8] and [Sw/8][4 planes][ncolp][bins][8], with
// Xp[q] / Yp[q] pointing at plane q of group 0 (only Xp[0] / Yp[0] are
// allocations); and Yh / Xh as the contractions' complex64 outputs.
struct FftBuffers {
    float2* Wf = nullptr;
    float2* Xh = nullptr;
    float2* Yh = nullptr;
    __nv_bfloat16* Wp[4] = {};
    __nv_bfloat16* Xp[4] = {};
    __nv_bfloat16* Yp[4] = {};
    int ncolp = 16;           // rows per bin of the Xp / Yp planes (columns padded to 16)
    void* cg = nullptr;
};

// One frame of a batch whose frames differ in shape (serving): the transforms
// find a column's frame through a column -> frame table, and the frame's
// columns col0 .. col0 + tiles_y * tiles_x - 1 are its tiles in row-major order.
struct FrameCols {
    const float* vsrc;  // forward transform input: volume [C][Ly][Lx]
    const float* rsrc;  // backward transform input: ratio [S][Ly][Lx]; null = all ones
    float* rcm;         // forward output: ratio [S][Ly][Lx]
    const float* ycm;   // data [S][Ly][Lx]
    float* rimg;        // forward output: ratio image [H][W] (or null)
    float* xcm;         // backward output [C][Ly][Lx]
    int Ly, Lx, tiles_x, col0;
};

// picks F (or uses force_F if non-zero) by a bandwidth / arithmetic cost model
// for `frames` frames, with the contraction on the CUDA cores (tc_products 0,
// FP32) or the tensor cores (2: BF16 PSF spectra, 3: split BF16); false if no
// plan fits (> 64 tiles, spectra too large, or more than 256 phases)
bool fft_plan_for(const Geo& g, FftPlan* p, int force_F = 0, int frames = 1, int tc_products = 0);

// half spectra of the packed PSF taps (W32 [T*T][Spad][Cpad]) into b.Wf or b.Wp
cudaError_t fft_init(const FftPlan& p, const Geo& g, const float* W32, const FftBuffers& b,
                     cudaStream_t st);
// ev (may be null): two events recorded after the transform and after the
// contraction, for per-kernel timing.
// forward projection of the channel-major volume vcm [C][Ly][Lx]; writes the
// image Hv to img_out [H][W] and / or r = y / (Hv + eps) to rcm [S][Ly][Lx]
// (and to rimg [H][W] in image layout when rimg is not null)
// nf frames share one transform / contraction launch: column col = frame *
// ntile + tile; per-frame arrays follow each other (frame strides C*Ly*Lx for
// channel-major volumes, S*Ly*Lx for polyphase images, H*W / Nz*H*W for images
// and stack-order volumes)
cudaError_t fft_forward(const FftPlan& p, const Geo& g, const FftBuffers& b, int nf, const float* vcm,
                        float* img_out, float* rcm, const float* ycm, float* rimg, float eps,
                        cudaStream_t st, cudaEvent_t* ev);
// backprojection of rcm [S][Ly][Lx] into xcm [C][Ly][Lx] and / or a stack-order volume
cudaError_t fft_backward(const FftPlan& p, const Geo& g, const FftBuffers& b, int nf, const float* rcm,
                         float* xcm, float* stack_out, cudaStream_t st, cudaEvent_t* ev);

// Serving: the forward / backward projection of the columns col0 .. col0+ncol-1
// of a frame table (frames of one PSF set, of different shapes); g supplies
// the set's N, S, C. ncol <= b.ncolp. The forward writes each frame's ratio
// (rcm, rimg); the backward reads each frame's rsrc (all ones where null) and
// writes its xcm.
cudaError_t fft_forward_tab(const FftPlan& p, const Geo& g, const FftBuffers& b, const FrameCols* fr,
                            const int* colf, int col0, int ncol, float eps, cudaStream_t st);
cudaError_t fft_backward_tab(const FftPlan& p, const Geo& g, const FftBuffers& b, const FrameCols* fr,
                             const int* colf, int col0, int ncol, cudaStream_t st);
// exact backprojection of one frame at the *n voxels of list (device count);
// rimg == null backprojects an all-ones image
cudaError_t launch_exact_bwd_dev(const int* list, const int* n, const float* rimg, const float* psf,
                                 const Geo& g, float* xcm, cudaStream_t st);
// list <- indices e < n with !(x[e] >= frac * max(0, max x)), *count <- their number
cudaError_t launch_low_list(const float* x, int64_t n, float frac, unsigned* mx, int* list, int* count,
                            cudaStream_t st);

cudaError_t launch_poly_volume_cm(const float* v, const Geo& g, float* vcm, cudaStream_t st);
cudaError_t launch_depoly_volume_cm(const float* vcm, const Geo& g, float* v, cudaStream_t st);
cudaError_t launch_poly_image_cm(const float* y, const Geo& g, float* ycm, cudaStream_t st);
cudaError_t launch_fill_cm(float* p, int64_t n, float val, cudaStream_t st);
cudaError_t launch_inv_cm(const float* x, int64_t n, float* inv, cudaStream_t st);
// exact backprojection of rimg [H][W] at the voxels list[0..n) (linear
// channel-major indices c*Ly*Lx + Iy*Lx + Ix), written into xcm; psf is the
// original [Nz][Nnum][Nnum][P][P] array
cudaError_t launch_exact_bwd(const int64_t* list, int64_t n, int nf, const float* rimg,
                             const float* psf, const Geo& g, float* xcm, cudaStream_t st);
int update_cm_blocks(const Geo& g);
// one flux partial per block: update_cm_blocks(g) per frame, frame-major
cudaError_t launch_update_cm(const float* vin, float* vout, const float* x, const float* inv,
                             const Geo& g, int nf, float* mip, double* flux_part, cudaStream_t st);

}  // namespace lfd
