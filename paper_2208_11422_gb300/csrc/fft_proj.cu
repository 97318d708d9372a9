// FFT variant of the light-field projections (FP32 throughout).
//
// In polyphase form both projections are multi-channel 2-D convolutions on the
// lenslet grid with kernels of T x T taps (lfd_internal.h):
//   forward   Hv[s]   = sum_c  Wp[.][s][c]  (*)  V[c]      (convolution)
//   backward  HtR[c]  = sum_s  Wp[.][s][c]  (x)  R[s]      (correlation)
// Overlap-save on tiles: an F x F patch (F = 32 or 64) holds B = F - 2h valid
// outputs per axis, so the grid is covered by tiles_y x tiles_x patches. Every
// (s, c) kernel is transformed once (at context creation) into its F x (F/2+1)
// half spectrum Wf[bin][s][c]. Per projection:
//   1. R2C transform of every input channel's patch of every tile,
//   2. per frequency bin a complex contraction over channels
//        forward  Yh[bin][tile][s] = sum_c Wf[bin][s][c]       Xh[bin][tile][c]
//        backward Xh[bin][tile][c] = sum_s conj(Wf[bin][s][c]) Yh[bin][tile][s]
//   3. C2R transform of every output channel's patch; the valid window is
//      [2h, F) for the convolution and [0, B) for the correlation.
// The ratio r = y / (Hv + eps) is fused into the forward's C2R store.
//
// Transforms are radix-2 in registers: each F-point 1-D transform is split by
// decimation in frequency over two lanes, each holding an F/2-point transform
// (F lanes per channel), with the channel's half spectrum staged in shared
// memory between the row and column passes. The contractions run on the
// tcgen05 tensor cores (split BF16 or BF16 PSF spectra, tc_cgemm.cu) or, for
// LFD_FP32, on the CUDA cores in FP32 (below), streaming the cached PSF
// spectra once per projection.
#include <algorithm>
#include <cmath>
#include <vector>

#include "fft_proj.h"
#include "tc_cgemm.h"

namespace lfd {
namespace {

__constant__ float2 c_tw[32];  // exp(-2 pi i k / 64), k < 32

template <int F>
struct FftSize {
    static constexpr int LOG = F == 64 ? 6 : 5;
    static constexpr int HF = F / 2;           // points of each lane's 1-D transform (F/2)
    static constexpr int H2 = F / 2 + 1;       // half-spectrum columns
    static constexpr int BINS = F * H2;
    // Threads per block. R2C: 512 (8 channels at F = 64, 16 at F = 32), so
    // that its outputs go out as whole 8-channel groups. C2R at F = 64: 4
    // channels in 256 threads and two blocks per SM (each 68 KB of half
    // spectra), so that one block's loads overlap the other's transforms
    // (1.84 -> 1.71 ms at the large frame; the R2C measured 1.70 -> 1.74 ms
    // that way); at F = 32, 512.
    static constexpr int R2C_THREADS = 512;
    static constexpr int C2R_THREADS = F == 64 ? 256 : 512;
    static constexpr int C2R_MINB = 512 / C2R_THREADS;  // blocks per SM (launch bounds)
    static constexpr int R2C_CH = R2C_THREADS / F;       // channels per block: F lanes each
    static constexpr int C2R_CH = C2R_THREADS / F;
    static constexpr int C2R_GCH = C2R_CH < 8 ? C2R_CH : 8;  // channels per input group item
};

__device__ __forceinline__ int brev_c(int i, int log) {
    int r = 0;
#pragma unroll
    for (int b = 0; b < 6; ++b)
        if (b < log) r |= ((i >> b) & 1) << (log - 1 - b);
    return r;
}

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }


// Radix-2 decimation-in-time FFT of N <= 64 points held in one thread's
// registers: a[] in bit-reversed order on entry, natural order on exit. One
// template instance per stage (LEN = 2, 4, ..., N) keeps every index a
// compile-time constant, so a[] stays in registers and each twiddle
// exp(-+2 pi i j / LEN) = c_tw[j * 64 / LEN] is a constant-bank operand; the
// factors 1 and -+i are applied without a multiply. INV: conjugate twiddles
// (no scaling).
template <int N, int LEN, bool INV>
__device__ __forceinline__ void fft_stage(float2 (&a)[N]) {
    constexpr int HALF = LEN / 2;
#pragma unroll
    for (int g = 0; g < N / LEN; ++g) {
#pragma unroll
        for (int j = 0; j < HALF; ++j) {
            const int i = g * LEN, tw = j * (64 / LEN);
            const float2 u = a[i + j], v = a[i + j + HALF];
            float2 t;
            if (tw == 0) {
                t = v;
            } else if (tw == 16) {  // exp(-i pi / 2) = -i (forward), +i (inverse)
                t = INV ? make_float2(-v.y, v.x) : make_float2(v.y, -v.x);
            } else {
                const float2 w = c_tw[tw];
                const float wy = INV ? -w.y : w.y;
                t = make_float2(fmaf(v.x, w.x, -v.y * wy), fmaf(v.x, wy, v.y * w.x));
            }
            a[i + j] = cadd(u, t);
            a[i + j + HALF] = csub(u, t);
        }
    }
    if constexpr (LEN < N) fft_stage<N, 2 * LEN, INV>(a);
}
template <int N, bool INV>
__device__ __forceinline__ void fft_reg(float2 (&a)[N]) {
    fft_stage<N, 2, INV>(a);
}

// Barrier of the F lanes of one channel of a transform block: a named
// barrier (id 1 + ch) over the channel's two warps when F = 64, the warp
// itself when F = 32; the channels of a block go through their phases
// independently.
template <int F>
__device__ __forceinline__ void chan_sync(int ch) {
    if constexpr (F >= 64) {
        // immediate barrier ids (one per channel of the block), so that the
        // block holds only the barriers it uses
        static_assert(FftSize<F>::R2C_CH <= 8 && FftSize<F>::C2R_CH <= 8, "one named barrier per channel");
        switch (ch) {
            case 0: asm volatile("bar.sync 1, %0;" ::"n"(F) : "memory"); break;
            case 1: asm volatile("bar.sync 2, %0;" ::"n"(F) : "memory"); break;
            case 2: asm volatile("bar.sync 3, %0;" ::"n"(F) : "memory"); break;
            case 3: asm volatile("bar.sync 4, %0;" ::"n"(F) : "memory"); break;
            case 4: asm volatile("bar.sync 5, %0;" ::"n"(F) : "memory"); break;
            case 5: asm volatile("bar.sync 6, %0;" ::"n"(F) : "memory"); break;
            case 6: asm volatile("bar.sync 7, %0;" ::"n"(F) : "memory"); break;
            default: asm volatile("bar.sync 8, %0;" ::"n"(F) : "memory"); break;
        }
    } else {
        __syncwarp();
    }
}

// v * exp(-+2 pi i n / F) for 0 <= n < F/2 (the decimation-in-frequency
// twiddle; INV: conjugate), a constant-bank operand when n is a constant
template <int F, bool INV>
__device__ __forceinline__ float2 twiddle(float2 v, int n) {
    const int tw = n * (64 / F);
    if (tw == 0) return v;
    if (tw == 16) return INV ? make_float2(-v.y, v.x) : make_float2(v.y, -v.x);
    const float2 w = c_tw[tw];
    const float wy = INV ? -w.y : w.y;
    return make_float2(fmaf(v.x, w.x, -v.y * wy), fmaf(v.x, wy, v.y * w.x));
}

// A source or destination is bound to one column (one tile of one frame)
// before a block's transforms: bind(col) returns a view of the tile's patch.
// Sources give rows of a channel's patch (row(c, r), then at(row, x) for the
// columns with col_ok(x)); destinations give output rows (row(c, i), then
// put(row, j, value)), so per-row address arithmetic is done once per row.

// patch view of a channel-major image [nch][Ly][Lx]: patch row r, column x is
// lenslet (y0 + r, x0 + x), zero outside the grid; base == null reads an
// all-ones image (used for H^T 1)
struct SrcRow {
    const float* p;  // patch column 0 of the row (valid only if ok)
    bool ok;
};
struct ImgView {
    const float* base;
    int Ly, Lx, y0, x0;
    __device__ bool col_ok(int x) const { return (unsigned)(x0 + x) < (unsigned)Lx; }
    __device__ SrcRow row(int c, int r) const {
        const int Iy = y0 + r;
        const bool ok = (unsigned)Iy < (unsigned)Ly;
        return SrcRow{base ? base + ((int64_t)c * Ly + (ok ? Iy : 0)) * Lx + x0 : nullptr, ok};
    }
    __device__ float at(const SrcRow& w, int x) const { return base ? w.p[x] : 1.f; }
};

// channel-major images, uniform frames; patch of tile (ty, tx) starts at
// lenslet (ty*B - h, tx*B - h); column col = frame * ntile + tile, frames
// fstride floats apart
struct ImgSrc {
    const float* img;
    int Ly, Lx, h, B, tiles_x, ntile;
    int64_t fstride;
    __device__ ImgView bind(int col) const {
        const int f = col / ntile, tile = col % ntile;
        const int ty = tile / tiles_x, tx = tile % tiles_x;
        return ImgView{img + f * fstride, Ly, Lx, ty * B - h, tx * B - h};
    }
};

// frames of different shapes (serving): column gc = col0 + col belongs to
// frame colf[gc]; vol selects the frame's volume or its ratio image
struct TabSrc {
    const FrameCols* fr;
    const int* colf;
    int col0, h, B;
    bool vol;
    __device__ ImgView bind(int col) const {
        const int gc = col0 + col;
        const FrameCols& d = fr[colf[gc]];
        const int tile = gc - d.col0, ty = tile / d.tiles_x, tx = tile % d.tiles_x;
        return ImgView{vol ? d.vsrc : d.rsrc, d.Ly, d.Lx, ty * B - h, tx * B - h};
    }
};

// packed PSF Wp[T*T][Spad][Cpad] read as one T x T kernel per (s, c); the
// "tile" index is s here, and tap (qy, qx) = (Dy + h, Dx + h)
struct TapView {
    const float* W;  // at phase s
    int T;
    int64_t tap_stride;
    __device__ bool col_ok(int x) const { return x < T; }
    __device__ SrcRow row(int c, int r) const {
        return SrcRow{W + (int64_t)(r < T ? r : 0) * T * tap_stride + c, r < T};
    }
    __device__ float at(const SrcRow& w, int x) const { return w.p[(int64_t)x * tap_stride]; }
};
struct TapSrc {
    const float* W;
    int T, Spad, Cpad;
    __device__ TapView bind(int s) const {
        return TapView{W + (int64_t)s * Cpad, T, (int64_t)Spad * Cpad};
    }
};

// spectrum outputs of the R2C transform: complex64, or BF16 planes
// (real hi, real lo, imag hi, imag lo; x = hi + lo) for the tensor cores.
// put8 writes channels c0 .. c0+7 of one bin and column that lie below the
// row length ld (c0 and ld are multiples of 4, so 4 or 8 of them) with
// 16-byte stores (8-byte for a group of 4 in the planes).
// BF16 planes of 8 complex values, two channels per 32-bit word (channel 2k
// in the low half): h[0] real hi, h[1] real lo, h[2] imag hi, h[3] imag lo,
// with hi = RN(x) and lo = RN(x - hi)
__device__ __forceinline__ void split8(const float2 (&v)[8], uint32_t (&h)[4][4]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float2 a = v[2 * k], b = v[2 * k + 1];
        const __nv_bfloat162 rh = __floats2bfloat162_rn(a.x, b.x), ih = __floats2bfloat162_rn(a.y, b.y);
        const float2 rb = __bfloat1622float2(rh), ib = __bfloat1622float2(ih);
        const __nv_bfloat162 rl = __floats2bfloat162_rn(a.x - rb.x, b.x - rb.y);
        const __nv_bfloat162 il = __floats2bfloat162_rn(a.y - ib.x, b.y - ib.y);
        h[0][k] = *reinterpret_cast<const uint32_t*>(&rh);
        h[1][k] = *reinterpret_cast<const uint32_t*>(&rl);
        h[2][k] = *reinterpret_cast<const uint32_t*>(&ih);
        h[3][k] = *reinterpret_cast<const uint32_t*>(&il);
    }
}

struct OutC64 {
    float2* p;
    int ntile, ld;
    __device__ void put8(int bin, int tile, int c0, const float2 (&v)[8]) const {
        float4* q = reinterpret_cast<float4*>(p + ((int64_t)bin * ntile + tile) * ld + c0);
        const int n4 = ld - c0 >= 8 ? 4 : 2;
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (k < n4) q[k] = make_float4(v[2 * k].x, v[2 * k].y, v[2 * k + 1].x, v[2 * k + 1].y);
    }
};
// (the lo planes p[1], p[3] may be null: BF16 PSF spectra keep only the hi planes)
struct OutPlanes {
    __nv_bfloat16* p[4];
    int ntile, ld;
    __device__ void put8(int bin, int tile, int c0, const float2 (&v)[8]) const {
        const int64_t o = ((int64_t)bin * ntile + tile) * ld + c0;
        uint32_t h[4][4];
        split8(v, h);
        if (ld - c0 >= 8) {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (p[q]) *reinterpret_cast<uint4*>(p[q] + o) = make_uint4(h[q][0], h[q][1], h[q][2], h[q][3]);
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (p[q]) *reinterpret_cast<uint2*>(p[q] + o) = make_uint2(h[q][0], h[q][1]);
        }
    }
};
// The transformed volume / ratio for the tensor-core contraction, in groups of
// 8 channels with the four planes of a group side by side:
// [g][plane q][col][bin][8] (g = channel / 8; p[q] points at plane q of group
// 0, groups are 4 ncolp bins x 8 values apart). One transform block writes,
// per plane, all bins of its channels of one column as one contiguous run;
// the contraction's TMA box (8 channels x 1 bin x n columns x 4 planes of
// each of its groups) lands in shared memory as [group][plane][column][8
// channels]: the canonical K-major layout without swizzle (8 x 16-byte core
// matrices) of one B operand whose N = 4n rows are the planes' columns.
struct OutPlanesG {
    __nv_bfloat16* p[4];
    int ncolp, bins;  // columns per group, bins per column
    __device__ void put8(int bin, int col, int c0, const float2 (&v)[8]) const {
        const int64_t o = (((int64_t)(c0 >> 3) * 4 * ncolp + col) * bins + bin) * 8;
        uint32_t h[4][4];
        split8(v, h);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            *reinterpret_cast<uint4*>(p[q] + o) = make_uint4(h[q][0], h[q][1], h[q][2], h[q][3]);
    }
};

// R2C 2-D transform of the F x F patches of FftSize<F>::R2C_CH channels of
// one tile; bin = fy*(F/2+1) + fx, out.put8 for every channel below ldc (zeros
// for channels >= nch). Each channel has F lanes, q = h * F/2 + l: every 1-D
// transform of F points is split over the two lanes (h = 0, 1) of one l by
// decimation in frequency: lane h = 0 transforms u[n] = x[n] + x[n + F/2] and
// obtains the even outputs X[2r], lane h = 1 transforms
// u[n] = (x[n] - x[n + F/2]) exp(-2 pi i n / F) and obtains the odd ones
// X[2r + 1]. The sums and differences are formed by the lanes that produce
// the values (so a lane reads only the F/2 values it transforms), and an
// F/2-point transform in registers per lane keeps the block at 512 threads.
//   load:    lane (h, l) loads columns l and l + F/2 of the patch rows
//            [h F/2, h F/2 + F/2) (coalesced across lanes) and stores their
//            sum and difference, Sx[r][l] and Dx[r][l];
//   rows:    lanes (h, l) transform rows l and l + F/2 packed as one complex
//            row z = p_l + i p_{l+F/2} (from Sx, or from Dx with the twiddle)
//            and separate the two half spectra (X[k] and X[F-k] have the same
//            parity, so each lane holds both); the real bins fx = 0 and F/2
//            of a row go to slot 0 as one complex value (bin 0 real part,
//            bin F/2 real part). For the columns they store, per bin, the
//            sum of rows l and l + F/2 in row l and their difference times
//            exp(-2 pi i l / F) in row l + F/2;
//   columns: lanes (h, l) transform column slot l (rows [h F/2, h F/2 + F/2)
//            hold their inputs), for l = 0 the packed real columns 0 and F/2,
//            which they separate afterwards.
// The half spectra stay in shared memory [channel][fy or row][fx], in place.
// Grid: x = channel group (fastest, so blocks running together fill adjacent
// parts of the same output rows), y = column.
template <int F, class Src, class Out>
__global__ void __launch_bounds__(FftSize<F>::R2C_THREADS, 1) k_fft_r2c(Src src, int nch, int ldc, Out out) {
    using Z = FftSize<F>;
    constexpr int HF = Z::HF, H2 = Z::H2, LOG = Z::LOG, CH = Z::R2C_CH, PS = HF + 1;
    extern __shared__ float2 sm[];
    const int ch = threadIdx.x / F, q = threadIdx.x % F;
    const int h = q / HF, l = q % HF;
    const int tile = blockIdx.y, c0 = blockIdx.x * CH, c = c0 + ch;
    const auto view = src.bind(tile);
    float2* R = sm + (size_t)ch * Z::BINS;          // [F][H2] half spectra
    float* Sx = reinterpret_cast<float*>(R);        // [F][PS] row-half sums (same space)
    float* Dx = Sx + F * PS;                        // [F][PS] row-half differences
    const bool on = c < nch;
    const float2 wl = c_tw[l * (64 / F)];           // exp(-2 pi i l / F), this lane's row twiddle
    {
        const bool ok0 = on && view.col_ok(l), ok1 = on && view.col_ok(l + HF);
        float t0[HF], t1[HF];
#pragma unroll
        for (int r = 0; r < HF; ++r) {
            const SrcRow w = view.row(on ? c : 0, h * HF + r);
            t0[r] = (ok0 && w.ok) ? view.at(w, l) : 0.f;
            t1[r] = (ok1 && w.ok) ? view.at(w, l + HF) : 0.f;
        }
#pragma unroll
        for (int r = 0; r < HF; ++r) {
            Sx[(h * HF + r) * PS + l] = t0[r] + t1[r];
            Dx[(h * HF + r) * PS + l] = t0[r] - t1[r];
        }
    }
    chan_sync<F>(ch);
    float2 a[HF];
    if (h == 0) {
#pragma unroll
        for (int n = 0; n < HF; ++n) a[brev_c(n, LOG - 1)] = make_float2(Sx[l * PS + n], Sx[(l + HF) * PS + n]);
    } else {
#pragma unroll
        for (int n = 0; n < HF; ++n)
            a[brev_c(n, LOG - 1)] = twiddle<F, false>(make_float2(Dx[l * PS + n], Dx[(l + HF) * PS + n]), n);
    }
    chan_sync<F>(ch);  // the half spectra below overwrite the row halves
    fft_reg<HF, false>(a);  // a[r] = Z[2r + h]
    // bin k of rows l (A) and l + HF (B): column inputs A + B and (A - B) w_l
    auto put = [&](int k, float2 A, float2 B) {
        R[l * H2 + k] = cadd(A, B);
        const float2 d = csub(A, B);
        R[(l + HF) * H2 + k] = make_float2(fmaf(d.x, wl.x, -d.y * wl.y), fmaf(d.x, wl.y, d.y * wl.x));
    };
    if (h == 0) {
        put(0, make_float2(a[0].x, a[HF / 2].x), make_float2(a[0].y, a[HF / 2].y));
#pragma unroll
        for (int r = 1; r < HF / 2; ++r) {
            const float2 z = a[r], m = a[HF - r];
            put(2 * r, make_float2(0.5f * (z.x + m.x), 0.5f * (z.y - m.y)),
                make_float2(0.5f * (z.y + m.y), 0.5f * (m.x - z.x)));
        }
    } else {
#pragma unroll
        for (int r = 0; r < HF / 2; ++r) {
            const float2 z = a[r], m = a[HF - 1 - r];
            put(2 * r + 1, make_float2(0.5f * (z.x + m.x), 0.5f * (z.y - m.y)),
                make_float2(0.5f * (z.y + m.y), 0.5f * (m.x - z.x)));
        }
    }
    chan_sync<F>(ch);
#pragma unroll
    for (int n = 0; n < HF; ++n) a[brev_c(n, LOG - 1)] = R[(h * HF + n) * H2 + l];
    chan_sync<F>(ch);  // every lane has read its column before the columns are rewritten
    fft_reg<HF, false>(a);  // a[s] = Y[2s + h]
    if (l == 0) {  // packed real columns 0 (real part) and F/2 (imaginary part); slot HF is free
#pragma unroll
        for (int s2 = 0; s2 < HF; ++s2) {
            const float2 z = a[s2], m = h == 0 ? a[(HF - s2) & (HF - 1)] : a[HF - 1 - s2];
            const int fy = 2 * s2 + h;
            R[fy * H2] = make_float2(0.5f * (z.x + m.x), 0.5f * (z.y - m.y));
            R[fy * H2 + HF] = make_float2(0.5f * (z.y + m.y), 0.5f * (m.x - z.x));
        }
    } else {
#pragma unroll
        for (int s2 = 0; s2 < HF; ++s2) R[(2 * s2 + h) * H2 + l] = a[s2];
    }
    __syncthreads();  // the output loop reads every channel of the block
    // every bin of 8 consecutive channels at a time
    static_assert(CH % 8 == 0, "whole 8-channel groups per block");
    for (int e = threadIdx.x; e < Z::BINS * (CH / 8); e += blockDim.x) {
        const int bin = e % Z::BINS, g = e / Z::BINS;
        if (c0 + 8 * g >= ldc) continue;
        float2 v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = sm[(size_t)(8 * g + k) * Z::BINS + bin];
        out.put8(bin, tile, c0 + 8 * g, v);
    }
}

// forward output view of one tile: Hv of polyphase channel s at output (i, j)
// of the tile = lenslet (y0 + i, x0 + j); optionally stored as an image
// [H][W] and / or turned into r = y / (Hv + eps)
struct HvView {
    float* img;        // [H][W] or null
    float* rcm;        // [S][Ly][Lx] ratio or null
    const float* ycm;  // [S][Ly][Lx]
    float* rimg;       // [H][W] ratio in image layout or null
    float eps;
    int N, W, Ly, Lx, y0, x0;
    struct Chan {
        int64_t pix, o;  // image index (column stride N) and channel-major index of output (y0, x0)
    };
    struct Row {
        int64_t pix, o;
        bool ok;
    };
    __device__ Chan chan(int s) const {
        return Chan{((int64_t)y0 * N + s / N) * W + (int64_t)x0 * N + s % N, ((int64_t)s * Ly + y0) * Lx + x0};
    }
    __device__ bool col_ok(int j) const { return x0 + j < Lx; }
    __device__ Row row(const Chan& ch, int i) const {
        return Row{ch.pix + (int64_t)i * N * W, ch.o + (int64_t)i * Lx, y0 + i < Ly};
    }
    __device__ void put(const Row& w, int j, float hv) const {
        const int64_t pix = w.pix + (int64_t)j * N;
        if (img) img[pix] = hv;
        if (rcm) {
            const int64_t o = w.o + j;
            const float den = hv + eps;
            const float r = den > 0.f ? ycm[o] / den : 0.f;
            rcm[o] = r;
            if (rimg) rimg[pix] = r;
        }
    }
};
struct HvDst {
    float* img;        // [frames][H][W] or null
    float* rcm;        // [frames][S][Ly][Lx] ratio or null
    const float* ycm;  // [frames][S][Ly][Lx]
    float* rimg;       // [frames][H][W] ratio in image layout or null
    float eps;
    int N, W, Ly, Lx, B, tiles_x, ntile;
    int64_t fs_cm, fs_img;  // frame strides
    __device__ HvView bind(int col) const {
        const int f = col / ntile, tile = col % ntile;
        const int ty = tile / tiles_x, tx = tile % tiles_x;
        const int64_t oc = f * fs_cm, oi = f * fs_img;
        return HvView{img ? img + oi : nullptr, rcm ? rcm + oc : nullptr, ycm ? ycm + oc : nullptr,
                      rimg ? rimg + oi : nullptr, eps, N, W, Ly, Lx, ty * B, tx * B};
    }
};
struct TabHvDst {
    const FrameCols* fr;
    const int* colf;
    int col0, N, B;
    float eps;
    __device__ HvView bind(int col) const {
        const int gc = col0 + col;
        const FrameCols& d = fr[colf[gc]];
        const int tile = gc - d.col0, ty = tile / d.tiles_x, tx = tile % d.tiles_x;
        return HvView{nullptr, d.rcm, d.ycm, d.rimg, eps, N, d.Lx * N, d.Ly, d.Lx, ty * B, tx * B};
    }
};

// backward output view of one tile: H^T r of channel c = (z, t) at output
// (i, j) = lenslet (y0 + i, x0 + j), into a channel-major volume and / or a
// stack-order volume [Nz][H][W]
struct VolView {
    float* cm;     // [C][Ly][Lx] or null
    float* stack;  // [Nz][H][W] or null
    int N, S, H, W, Ly, Lx, y0, x0;
    struct Chan {
        int64_t cm, st;  // channel-major index and stack index (column stride N) of output (y0, x0)
    };
    struct Row {
        int64_t cm, st;
        bool ok;
    };
    __device__ Chan chan(int c) const {
        const int z = c / S, t = c % S;
        return Chan{((int64_t)c * Ly + y0) * Lx + x0,
                    ((int64_t)z * H + (int64_t)y0 * N + t / N) * W + (int64_t)x0 * N + t % N};
    }
    __device__ bool col_ok(int j) const { return x0 + j < Lx; }
    __device__ Row row(const Chan& ch, int i) const {
        return Row{ch.cm + (int64_t)i * Lx, ch.st + (int64_t)i * N * W, y0 + i < Ly};
    }
    __device__ void put(const Row& w, int j, float x) const {
        if (cm) cm[w.cm + j] = x;
        if (stack) stack[w.st + (int64_t)j * N] = x;
    }
};
struct VolDst {
    float* cm;     // [frames][C][Ly][Lx] or null
    float* stack;  // [frames][Nz][H][W] or null
    int N, S, H, W, Ly, Lx, B, tiles_x, ntile;
    int64_t fs_cm, fs_stack;  // frame strides
    __device__ VolView bind(int col) const {
        const int f = col / ntile, tile = col % ntile;
        const int ty = tile / tiles_x, tx = tile % tiles_x;
        return VolView{cm ? cm + f * fs_cm : nullptr, stack ? stack + f * fs_stack : nullptr,
                       N, S, H, W, Ly, Lx, ty * B, tx * B};
    }
};
struct TabVolDst {
    const FrameCols* fr;
    const int* colf;
    int col0, N, S, B;
    __device__ VolView bind(int col) const {
        const int gc = col0 + col;
        const FrameCols& d = fr[colf[gc]];
        const int tile = gc - d.col0, ty = tile / d.tiles_x, tx = tile % d.tiles_x;
        return VolView{d.xcm, nullptr, N, S, d.Ly * N, d.Lx * N, d.Ly, d.Lx, ty * B, tx * B};
    }
};

// C2R 2-D transform of FftSize<F>::C2R_CH channels of one tile: rows and
// columns [off, off + B) of the real result, times `scale`, go to dst. Each
// channel has F lanes, q = h * F/2 + l, and every 1-D transform is split over
// the two lanes (h = 0, 1) of one l by decimation in frequency (as in the
// R2C, with conjugate twiddles):
//   columns: lanes (h, l), l >= 1, inverse-transform column fx = l; for l = 0
//            they transform columns 0 and F/2 (whose inverses are real) packed
//            as one and leave both results in slot 0 (real part: column 0,
//            imaginary part: column F/2);
//   rows:    lanes (h, i), i < B/2, inverse-transform output rows off+i and
//            off+i+B/2 packed as one complex row (each row's spectrum
//            extended by conjugate symmetry); the outputs go through shared
//            memory so that dst sees consecutive j across lanes, one output
//            row at a time.
// Input (LAYOUT): 0, [BINS][ntile][ldc] (CUDA-core contraction); the
// tensor-core contraction's group-major outputs, 1 [ldc/8][ntile][BINS][8]
// (forward) or 2 [ldc/8][BINS][ntile][8] (adjoint).
// Grid: x = column, y = channel group (the blocks of one group that run
// together read the columns of each bin together).
template <int F, class Dst, int LAYOUT>
__global__ void __launch_bounds__(FftSize<F>::C2R_THREADS, FftSize<F>::C2R_MINB) k_fft_c2r(const float2* __restrict__ in, int nch,
                                                                  int ldc, int ntile, int off, int B,
                                                                  float scale, Dst dst) {
    using Z = FftSize<F>;
    constexpr int HF = Z::HF, H2 = Z::H2, LOG = Z::LOG, CH = Z::C2R_CH;
    extern __shared__ float2 sm[];
    const int ch = threadIdx.x / F, q = threadIdx.x % F;
    const int h = q / HF, l = q % HF;
    const int tile = blockIdx.x, c0 = blockIdx.y * CH, c = c0 + ch;
    const auto view = dst.bind(tile);
    // spectra of GCH (8, or the block's 4) consecutive channels per bin (one
    // thread reads them with 16-byte loads) for the bins (fy, fx) and
    // (fy + F/2, fx), stored into [channel][bin] as the column transform's
    // inputs: their sum in row fy and their difference times exp(2 pi i fy / F)
    // in row fy + F/2
    // All of a thread's loads are issued before the first is used (their
    // latency is paid once per block, not once per item). A sub-item is one
    // 16-byte piece (two channels) of an item's two bins; the lanes of a warp
    // take the pieces of 32 / PIECES items, lane L piece L / (32 / PIECES), so
    // a warp's load touches as many 32-byte sectors as items (not lanes) and
    // its 8-byte shared-memory stores split into half-warps without bank
    // conflicts.
    constexpr int GCH = Z::C2R_GCH, PIECES = GCH / 2, IPW = 32 / PIECES;
    static_assert(CH % GCH == 0 && 8 % GCH == 0, "whole channel groups per block");
    constexpr int NITEM = HF * H2 * (CH / GCH), NSUB = NITEM * PIECES;
    static_assert(NSUB % 32 == 0, "whole warps of sub-items");
    constexpr int NIT = (NSUB + Z::C2R_THREADS - 1) / Z::C2R_THREADS;
    {
        float4 w0[NIT], w1[NIT];
#pragma unroll
        for (int it = 0; it < NIT; ++it) {
            const int sub = threadIdx.x + it * Z::C2R_THREADS;
            const int e = (sub >> 5) * IPW + (sub & 31) % IPW, k = (sub & 31) / IPW;
            const int fx = e % H2, fy = (e / H2) % HF, g = e / (H2 * HF), cg = c0 + GCH * g;
            const int b0 = fy * H2 + fx, b1 = b0 + HF * H2;
            w0[it] = w1[it] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (sub < NSUB && cg < ldc) {  // ldc is a multiple of 8 (run_c2r checks)
                const float2* base =
                    LAYOUT == 1   ? in + ((int64_t)(cg >> 3) * ntile + tile) * Z::BINS * 8 + (cg & 7)
                    : LAYOUT == 2 ? in + ((int64_t)(cg >> 3) * Z::BINS * ntile + tile) * 8 + (cg & 7)
                                  : in + (int64_t)tile * ldc + cg;
                const int64_t bstride = LAYOUT == 1 ? 8 : LAYOUT == 2 ? (int64_t)ntile * 8
                                                                      : (int64_t)ntile * ldc;  // float2 between bins
                w0[it] = reinterpret_cast<const float4*>(base + b0 * bstride)[k];
                w1[it] = reinterpret_cast<const float4*>(base + b1 * bstride)[k];
            }
        }
#pragma unroll
        for (int it = 0; it < NIT; ++it) {
            const int sub = threadIdx.x + it * Z::C2R_THREADS;
            const int e = (sub >> 5) * IPW + (sub & 31) % IPW, k = (sub & 31) / IPW;
            if (sub >= NSUB) break;
            const int fx = e % H2, fy = (e / H2) % HF, g = e / (H2 * HF);
            const int b0 = fy * H2 + fx, b1 = b0 + HF * H2;
            const float2 w = c_tw[fy * (64 / F)];  // conjugated below
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const float4 a = w0[it], bb = w1[it];
                const float2 v0 = j ? make_float2(a.z, a.w) : make_float2(a.x, a.y);
                const float2 v1 = j ? make_float2(bb.z, bb.w) : make_float2(bb.x, bb.y);
                float2* dst = sm + (size_t)(GCH * g + 2 * k + j) * Z::BINS;
                dst[b0] = cadd(v0, v1);
                const float2 d = csub(v0, v1);
                dst[b1] = make_float2(fmaf(d.x, w.x, d.y * w.y), fmaf(d.y, w.x, -d.x * w.y));
            }
        }
    }
    __syncthreads();
    float2* R = sm + (size_t)ch * Z::BINS;  // [F][H2]
    float2 a[HF];
    // column slot l, rows [h F/2, h F/2 + F/2) (slot 0: columns 0 and F/2 packed)
#pragma unroll
    for (int n = 0; n < HF; ++n) {
        const int r = h * HF + n;
        float2 y;
        if (l == 0) {
            const float2 x0 = R[r * H2], xh = R[r * H2 + HF];
            y = make_float2(x0.x - xh.y, x0.y + xh.x);
        } else {
            y = R[r * H2 + l];
        }
        a[brev_c(n, LOG - 1)] = y;
    }
    chan_sync<F>(ch);  // every lane has read its column before the columns are rewritten
    fft_reg<HF, true>(a);  // a[s] = column value at row 2s + h
#pragma unroll
    for (int s2 = 0; s2 < HF; ++s2) R[(2 * s2 + h) * H2 + l] = a[s2];
    chan_sync<F>(ch);
    const int hb = B >> 1, ob = B + 1;  // row pairs; staged row stride
    float* O = reinterpret_cast<float*>(R);
    if (l < hb) {
        const float2* r1 = R + (off + l) * H2;
        const float2* r2 = R + (off + l + hb) * H2;
        // the packed row pair's spectrum Q[k] = R1[k] + i R2[k] over all F bins
        auto Q = [&](int k) -> float2 {
            if (k == 0) return make_float2(r1[0].x, r2[0].x);
            if (k == HF) return make_float2(r1[0].y, r2[0].y);
            float2 t1, t2;
            if (k < HF) {
                t1 = r1[k];
                t2 = r2[k];
            } else {
                t1 = r1[F - k];
                t2 = r2[F - k];
                t1.y = -t1.y;
                t2.y = -t2.y;
            }
            return make_float2(t1.x - t2.y, t1.y + t2.x);
        };
        if (h == 0) {
#pragma unroll
            for (int n = 0; n < HF; ++n) a[brev_c(n, LOG - 1)] = cadd(Q(n), Q(n + HF));
        } else {
#pragma unroll
            for (int n = 0; n < HF; ++n) a[brev_c(n, LOG - 1)] = twiddle<F, true>(csub(Q(n), Q(n + HF)), n);
        }
    }
    chan_sync<F>(ch);  // every lane has read its rows before R is reused for the outputs
    if (l < hb) {
        fft_reg<HF, true>(a);  // a[s] = row(off+l)[x] + i row(off+l+hb)[x], x = 2s + h
#pragma unroll
        for (int s2 = 0; s2 < HF; ++s2) {
            const int j = 2 * s2 + h - off;
            if (j >= 0 && j < B) {
                O[l * ob + j] = a[s2].x * scale;
                O[(l + hb) * ob + j] = a[s2].y * scale;
            }
        }
    }
    chan_sync<F>(ch);
    if (c < nch) {
        // lane q takes output column j = q of one row at a time (B < F)
        const auto chn = view.chan(c);
        const bool ok = q < B && view.col_ok(q);
        for (int i = 0; i < B; ++i) {
            const auto w = view.row(chn, i);
            if (!w.ok) break;  // the rows below are outside the grid as well
            if (ok) view.put(w, q, O[i * ob + q]);
        }
    }
}

// forward contraction: Yh[bin][t][s] = sum_c Wf[bin][s][c] Xh[bin][t][c].
// One block per bin, one thread per phase s holding all tiles (<= 16) in
// registers. Each thread streams its own row of Wf straight from global memory
// (32-byte loads, prefetched one step ahead); the tiles' spectra for the
// current 64 channels are broadcast from shared memory.
constexpr int kFC = 64;  // channels per shared-memory chunk
template <int NT>
__global__ void __launch_bounds__(256) k_contract_fwd(const float2* __restrict__ Wf,
                                                      const float2* __restrict__ Xh,
                                                      float2* __restrict__ Yh, int S, int Sf,
                                                      int C, int Cf, int ntile, int col0, int ncol) {
    __shared__ __align__(16) float2 Xs[kFC][NT];
    const int bin = blockIdx.x;
    const int s = threadIdx.x;
    const bool active = s < S;
    const float2* wrow = Wf + ((int64_t)bin * S + (active ? s : 0)) * Cf;
    const float2* Xb = Xh + ((int64_t)bin * ncol + col0) * Cf;
    float ar[NT], ai[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) ar[t] = ai[t] = 0.f;
    for (int k0 = 0; k0 < C; k0 += kFC) {
        __syncthreads();
        for (int e = threadIdx.x; e < kFC * NT; e += blockDim.x) {
            const int t = e / kFC, k = e % kFC, c = k0 + k;
            Xs[k][t] = (t < ntile && c < C) ? Xb[(int64_t)t * Cf + c] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        if (!active) continue;
        const int kn = min(kFC, C - k0);
        float4 w01 = make_float4(0.f, 0.f, 0.f, 0.f), w23 = w01;
        if (kn >= 4) {
            w01 = *reinterpret_cast<const float4*>(wrow + k0);
            w23 = *reinterpret_cast<const float4*>(wrow + k0 + 2);
        }
        for (int k = 0; k < kn; k += 4) {
            float4 n01 = make_float4(0.f, 0.f, 0.f, 0.f), n23 = n01;
            if (k + 8 <= kn) {  // prefetch the next 4 channels
                n01 = *reinterpret_cast<const float4*>(wrow + k0 + k + 4);
                n23 = *reinterpret_cast<const float4*>(wrow + k0 + k + 6);
            }
            float2 w[4] = {make_float2(w01.x, w01.y), make_float2(w01.z, w01.w),
                           make_float2(w23.x, w23.y), make_float2(w23.z, w23.w)};
            if (k + 4 > kn) {  // ragged end of C (C % 4 != 0)
                for (int q = 0; q < 4; ++q)
                    w[q] = k + q < kn ? wrow[k0 + k + q] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
#pragma unroll
                for (int t = 0; t < NT; ++t) {
                    const float2 x = Xs[k + q][t];
                    ar[t] = fmaf(w[q].x, x.x, fmaf(-w[q].y, x.y, ar[t]));
                    ai[t] = fmaf(w[q].x, x.y, fmaf(w[q].y, x.x, ai[t]));
                }
            }
            w01 = n01;
            w23 = n23;
        }
    }
    if (!active) return;
    float2* Yb = Yh + ((int64_t)bin * ncol + col0) * Sf;
#pragma unroll
    for (int t = 0; t < NT; ++t)
        if (t < ntile) Yb[(int64_t)t * Sf + s] = make_float2(ar[t], ai[t]);
}

// backward contraction: Xh[bin][t][c] = sum_s conj(Wf[bin][s][c]) Yh[bin][t][s].
// One block per (bin, 512 channels), two channels per thread, all tiles in
// registers; Wf rows are read coalesced, Yh[bin] sits in shared memory.
template <int NT>
__global__ void __launch_bounds__(256) k_contract_adj(const float2* __restrict__ Wf,
                                                      const float2* __restrict__ Yh,
                                                      float2* __restrict__ Xh, int S, int Sf,
                                                      int C, int Cf, int ntile, int col0, int ncol) {
    extern __shared__ float2 Ys[];  // [S][NT]
    const int bin = blockIdx.x;
    const int c = blockIdx.y * 512 + 2 * threadIdx.x;
    const float2* Wb = Wf + (int64_t)bin * S * Cf;
    const float2* Yb = Yh + ((int64_t)bin * ncol + col0) * Sf;
    for (int e = threadIdx.x; e < S * NT; e += blockDim.x) {
        const int sidx = e / NT, t = e % NT;
        Ys[e] = t < ntile ? Yb[(int64_t)t * Sf + sidx] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    if (c >= Cf) return;
    float ar0[NT], ai0[NT], ar1[NT], ai1[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) ar0[t] = ai0[t] = ar1[t] = ai1[t] = 0.f;
    float4 w = *reinterpret_cast<const float4*>(Wb + c);
    for (int sidx = 0; sidx < S; ++sidx) {
        float4 wn = make_float4(0.f, 0.f, 0.f, 0.f);
        if (sidx + 1 < S) wn = *reinterpret_cast<const float4*>(Wb + (int64_t)(sidx + 1) * Cf + c);
        const float2* yrow = Ys + sidx * NT;
#pragma unroll
        for (int t = 0; t < NT; ++t) {  // conj(w) * y
            const float2 y = yrow[t];
            ar0[t] = fmaf(w.x, y.x, fmaf(w.y, y.y, ar0[t]));
            ai0[t] = fmaf(w.x, y.y, fmaf(-w.y, y.x, ai0[t]));
            ar1[t] = fmaf(w.z, y.x, fmaf(w.w, y.y, ar1[t]));
            ai1[t] = fmaf(w.z, y.y, fmaf(-w.w, y.x, ai1[t]));
        }
        w = wn;
    }
    float2* Xb = Xh + ((int64_t)bin * ncol + col0) * Cf;
#pragma unroll
    for (int t = 0; t < NT; ++t)
        if (t < ntile)
            *reinterpret_cast<float4*>(Xb + (int64_t)t * Cf + c) = make_float4(ar0[t], ai0[t], ar1[t], ai1[t]);
}

template <int NT>
cudaError_t run_contract_fwd(const FftPlan& p, const Geo& g, const float2* Wf, const float2* Xh,
                             float2* Yh, int col0, int ngrp, int ncol, cudaStream_t st) {
    k_contract_fwd<NT><<<p.bins, 256, 0, st>>>(Wf, Xh, Yh, g.S, p.Sf, g.C, p.Cf, ngrp, col0, ncol);
    count_launch();
    return cudaGetLastError();
}
template <int NT>
cudaError_t run_contract_adj(const FftPlan& p, const Geo& g, const float2* Wf, const float2* Yh,
                             float2* Xh, int col0, int ngrp, int ncol, cudaStream_t st) {
    const size_t smem = sizeof(float2) * (size_t)g.S * NT;
    cudaError_t e = cudaFuncSetAttribute(k_contract_adj<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)p.bins, (unsigned)((p.Cf + 511) / 512));
    k_contract_adj<NT><<<grid, 256, smem, st>>>(Wf, Yh, Xh, g.S, p.Sf, g.C, p.Cf, ngrp, col0, ncol);
    count_launch();
    return cudaGetLastError();
}

// FP32 contractions over all ncol columns, in groups of at most 16 (each
// group streams the spectra once)
cudaError_t contract_fwd_all(const FftPlan& p, const Geo& g, const float2* Wf, const float2* Xh,
                             float2* Yh, int ncol, cudaStream_t st) {
    for (int c0 = 0; c0 < ncol; c0 += 16) {
        const int n = std::min(16, ncol - c0);
        cudaError_t e = n <= 1 ? run_contract_fwd<1>(p, g, Wf, Xh, Yh, c0, n, ncol, st)
                        : n <= 4 ? run_contract_fwd<4>(p, g, Wf, Xh, Yh, c0, n, ncol, st)
                        : n <= 9 ? run_contract_fwd<9>(p, g, Wf, Xh, Yh, c0, n, ncol, st)
                                 : run_contract_fwd<16>(p, g, Wf, Xh, Yh, c0, n, ncol, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}
cudaError_t contract_adj_all(const FftPlan& p, const Geo& g, const float2* Wf, const float2* Yh,
                             float2* Xh, int ncol, cudaStream_t st) {
    for (int c0 = 0; c0 < ncol; c0 += 16) {
        const int n = std::min(16, ncol - c0);
        cudaError_t e = n <= 1 ? run_contract_adj<1>(p, g, Wf, Yh, Xh, c0, n, ncol, st)
                        : n <= 4 ? run_contract_adj<4>(p, g, Wf, Yh, Xh, c0, n, ncol, st)
                        : n <= 9 ? run_contract_adj<9>(p, g, Wf, Yh, Xh, c0, n, ncol, st)
                                 : run_contract_adj<16>(p, g, Wf, Yh, Xh, c0, n, ncol, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Exact backprojection at listed voxels, by direct summation over each voxel's
// PSF window clipped to the sensor (one warp per voxel, FP32 products, one
// partial sum per PSF row):
//   X[c][Iy][Ix] = sum_{i,j} r[i][j] K[z][ty][tx][i - i' + c0][j - j' + c0]
// with c = (z, t = ty*N + tx), i' = Iy*N + ty, j' = Ix*N + tx. The FFT variant
// uses it for voxels whose sensitivity H^T 1 is so small that the transforms'
// absolute error floor would dominate their update.
// exact H^T r at channel-major voxel idx of one frame; rimg == null reads an
// all-ones image (H^T 1); one warp, result valid in every lane
__device__ float exact_bwd_voxel(int64_t idx, const float* __restrict__ rimg,
                                 const float* __restrict__ psf, const Geo& g) {
    const int lane = threadIdx.x & 31;
    const int64_t L2 = (int64_t)g.Ly * g.Lx;
    const int c0 = (g.P - 1) / 2;
    const int c = (int)(idx / L2);
    const int64_t l = idx % L2;
    const int Iy = (int)(l / g.Lx), Ix = (int)(l % g.Lx);
    const int z = c / g.S, t = c % g.S, ty = t / g.N, tx = t % g.N;
    const int ip = Iy * g.N + ty, jp = Ix * g.N + tx;
    const float* K = psf + (((int64_t)z * g.N + ty) * g.N + tx) * g.P * g.P;
    const int mi0 = max(0, c0 - ip), mi1 = min(g.P, g.H + c0 - ip);
    const int mj0 = max(0, c0 - jp), mj1 = min(g.P, g.W + c0 - jp);
    // lanes along the window's columns; a window narrower than 32 columns
    // takes 32 / width rows per step
    const int ncl = max(0, mj1 - mj0);
    const int rps = ncl >= 32 || ncl == 0 ? 1 : 32 / ncl;   // rows per step
    const int dr = ncl >= 32 ? 0 : lane / max(ncl, 1), cc = ncl >= 32 ? lane : lane % max(ncl, 1);
    const bool act = ncl >= 32 || lane < rps * ncl;
    const float* rr = rimg ? rimg + (int64_t)(ip - c0) * g.W + (jp - c0) : nullptr;
    float acc = 0.f;
    if (act) {
#pragma unroll 4
        for (int mi = mi0 + dr; mi < mi1; mi += rps) {
            const float* kk = K + (int64_t)mi * g.P;
            if (rr) {
                const float* rw = rr + (int64_t)mi * g.W;
                for (int mj = mj0 + cc; mj < mj1; mj += 32) acc = fmaf(rw[mj], kk[mj], acc);
            } else {
                for (int mj = mj0 + cc; mj < mj1; mj += 32) acc += kk[mj];
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    return acc;
}

__global__ void k_exact_bwd(const int64_t* __restrict__ list, int64_t n, int nf,
                            const float* __restrict__ rimg, const float* __restrict__ psf, Geo g,
                            float* __restrict__ xcm) {
    const int64_t L2 = (int64_t)g.Ly * g.Lx;
    for (int64_t qq = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; qq < n * nf;
         qq += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int f = (int)(qq / n);
        const int64_t idx = list[qq % n];
        const float acc = exact_bwd_voxel(idx, rimg + (int64_t)f * g.H * g.W, psf, g);
        if ((threadIdx.x & 31) == 0) xcm[(int64_t)f * g.C * L2 + idx] = acc;
    }
}

// the same for one frame whose voxel list and its length live on the device
__global__ void k_exact_bwd_dev(const int* __restrict__ list, const int* __restrict__ n,
                                const float* __restrict__ rimg, const float* __restrict__ psf, Geo g,
                                float* __restrict__ xcm) {
    const int cnt = *n;
    for (int64_t qq = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; qq < cnt;
         qq += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t idx = list[qq];
        const float acc = exact_bwd_voxel(idx, rimg, psf, g);
        if ((threadIdx.x & 31) == 0) xcm[idx] = acc;
    }
}

// largest value of x[0..n) (clamped at 0) into *mx (zeroed beforehand); the
// bit patterns of non-negative floats order like the floats themselves
__global__ void k_max_nonneg(const float* __restrict__ x, int64_t n, unsigned* __restrict__ mx) {
    float m = 0.f;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, x[e]);
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(mx, __float_as_uint(m));
}

// appends every index with !(x >= frac * max) to list (in no particular order)
__global__ void k_low_list(const float* __restrict__ x, int64_t n, const unsigned* __restrict__ mx,
                           float frac, int* __restrict__ list, int* __restrict__ count) {
    const float thr = frac * __uint_as_float(*mx);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x)
        if (!(x[e] >= thr)) list[atomicAdd(count, 1)] = (int)e;
}

// ------------------------------------------------ layout and update kernels --
// Stack-order planes <-> channel-major polyphase planes:
//   img[z][Iy*N+ty][Ix*N+tx]  <->  cm[z*S + ty*N + tx][Iy][Ix]
// (a volume has Nz planes, an image one). One block per image row y = Iy*N
// + ty of one plane: the row goes through shared memory, so the image side is
// read / written as one contiguous row and the channel side as N runs of Lx
// values (the row's lenslets of the channels (ty, tx)), a warp per tx and 32
// lenslets per access (the shared-memory stride N is odd, so these accesses
// are free of bank conflicts). Blocks of 32 lenslets of one lenslet row (N
// rows at a time, 128-byte channel runs) measured 2.3x slower at the large
// frame, and per-element index divisions cost as much again.
// Grid: x = image row, y = plane.
__global__ void __launch_bounds__(256) k_to_cm(const float* __restrict__ img, Geo g, float* __restrict__ cm) {
    extern __shared__ float row[];  // [W]
    const int y = blockIdx.x, z = blockIdx.y;
    const int Iy = y / g.N, ty = y - Iy * g.N;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const float* src = img + ((int64_t)z * g.H + y) * g.W;
    for (int x = threadIdx.x; x < g.W; x += blockDim.x) row[x] = src[x];
    __syncthreads();
    const int64_t L2 = (int64_t)g.Ly * g.Lx;
    float* dst = cm + ((int64_t)z * g.S + (int64_t)ty * g.N) * L2 + (int64_t)Iy * g.Lx;
    for (int tx = warp; tx < g.N; tx += nw)
        for (int Ix = lane; Ix < g.Lx; Ix += 32) dst[tx * L2 + Ix] = row[Ix * g.N + tx];
}
__global__ void __launch_bounds__(256) k_from_cm(const float* __restrict__ cm, Geo g, float* __restrict__ img) {
    extern __shared__ float row[];  // [W]
    const int y = blockIdx.x, z = blockIdx.y;
    const int Iy = y / g.N, ty = y - Iy * g.N;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int64_t L2 = (int64_t)g.Ly * g.Lx;
    const float* src = cm + ((int64_t)z * g.S + (int64_t)ty * g.N) * L2 + (int64_t)Iy * g.Lx;
    for (int tx = warp; tx < g.N; tx += nw)
        for (int Ix = lane; Ix < g.Lx; Ix += 32) row[Ix * g.N + tx] = src[tx * L2 + Ix];
    __syncthreads();
    float* dst = img + ((int64_t)z * g.H + y) * g.W;
    for (int x = threadIdx.x; x < g.W; x += blockDim.x) dst[x] = row[x];
}
__global__ void k_fill_cm(float* __restrict__ p, int64_t n, float val) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x)
        p[e] = val;
}
__global__ void k_inv_cm(const float* __restrict__ x, int64_t n, float* __restrict__ inv) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x)
        inv[e] = x[e] > 0.f ? 1.0f / x[e] : 0.f;
}

// RL update on channel-major volumes; thread per (phase t, lenslet), walking
// the depths: v_new = max(0, v * x * inv) (NaN -> 0, 0 where H^T 1 = 0), the
// z-maximum of v_new for its pixel, and the flux sum(v * x) where H^T 1 > 0
// (compensated FP32 over the thread's depths, FP64 across threads). The loads
// of 16 depths are issued together.
constexpr int kUpdBatch = 16;
__global__ void __launch_bounds__(256) k_update_cm(const float* __restrict__ vin, float* __restrict__ vout,
                                                   const float* __restrict__ x, const float* __restrict__ inv,
                                                   Geo g, float* __restrict__ mip,
                                                   double* __restrict__ flux_part) {
    __shared__ double red[8];
    const int64_t L2 = (int64_t)g.Ly * g.Lx, total = (int64_t)g.S * L2;
    {  // frame blockIdx.y: shift the per-frame arrays (H^T 1 is shared)
        const int64_t fv = (int64_t)blockIdx.y * g.C * L2;
        vin += fv;
        vout += fv;
        x += fv;
        mip += (int64_t)blockIdx.y * g.H * g.W;
        flux_part += (int64_t)blockIdx.y * gridDim.x;
    }
    double flux = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int t = (int)(e / L2);
        const int64_t l = e % L2;
        float mx = 0.f, fs = 0.f, fc = 0.f;
        const int64_t zs = (int64_t)g.S * L2;  // stride between depths
        const int64_t o0 = (int64_t)t * L2 + l;
        auto step = [&](float ivq, float voq, float xq, int64_t o) {
            float vn = 0.f;
            if (ivq > 0.f) {
                const float vx = voq * xq;
                vn = vx * ivq;
                kahan_add(fs, fc, vx);
            }
            vn = vn > 0.f ? vn : 0.f;
            vout[o] = vn;
            mx = fmaxf(mx, vn);
        };
        int z = 0;
        for (; z + kUpdBatch <= g.Nz; z += kUpdBatch) {
            float iv[kUpdBatch], vo[kUpdBatch], xx[kUpdBatch];
#pragma unroll
            for (int q = 0; q < kUpdBatch; ++q) {
                const int64_t o = o0 + (z + q) * zs;
                iv[q] = inv[o];
                vo[q] = vin[o];
                xx[q] = x[o];
            }
#pragma unroll
            for (int q = 0; q < kUpdBatch; ++q) step(iv[q], vo[q], xx[q], o0 + (z + q) * zs);
        }
        for (; z < g.Nz; ++z) {
            const int64_t o = o0 + z * zs;
            step(inv[o], vin[o], x[o], o);
        }
        const int Iy = (int)(l / g.Lx), Ix = (int)(l % g.Lx);
        mip[((int64_t)Iy * g.N + t / g.N) * g.W + (int64_t)Ix * g.N + t % g.N] = mx;
        flux += (double)fs - (double)fc;
    }
    for (int o = 16; o > 0; o >>= 1) flux += __shfl_xor_sync(0xffffffffu, flux, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = flux;
    __syncthreads();
    if (threadIdx.x == 0) {
        double f = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) f += red[i];
        flux_part[blockIdx.x] = f;
    }
}

inline int grid_for(int64_t n, int cap = 152 * 16) {
    int64_t b = (n + 255) / 256;
    if (b < 1) b = 1;
    return (int)(b < cap ? b : cap);
}

template <int F>
size_t fft_smem(bool r2c) {
    return sizeof(float2) * (size_t)(r2c ? FftSize<F>::R2C_CH : FftSize<F>::C2R_CH) * FftSize<F>::BINS;
}

bool g_tw_ready[64] = {};

cudaError_t upload_twiddles() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && g_tw_ready[dev]) return cudaSuccess;
    float2 tw[32];
    const double pi = 3.14159265358979323846;
    for (int k = 0; k < 32; ++k)
        tw[k] = make_float2((float)std::cos(2.0 * pi * k / 64.0), (float)-std::sin(2.0 * pi * k / 64.0));
    e = cudaMemcpyToSymbol(c_tw, tw, sizeof(tw));
    if (e == cudaSuccess && dev >= 0 && dev < 64) g_tw_ready[dev] = true;
    return e;
}

template <int F, class Src, class Out>
cudaError_t run_r2c(Src src, int nch, int ldc, int ntile, Out out, cudaStream_t st) {
    const size_t smem = fft_smem<F>(true);
    cudaError_t e = cudaFuncSetAttribute(k_fft_r2c<F, Src, Out>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((ldc + FftSize<F>::R2C_CH - 1) / FftSize<F>::R2C_CH), (unsigned)ntile);
    k_fft_r2c<F, Src, Out><<<grid, FftSize<F>::R2C_THREADS, smem, st>>>(src, nch, ldc, out);
    count_launch();
    return cudaGetLastError();
}

// R2C into complex64 (FP32 contraction) or BF16 planes (tensor-core contraction)
template <class Src>
cudaError_t r2c_any(const FftPlan& p, Src src, int nch, int ldc, int ntile, float2* c64,
                    __nv_bfloat16* const* planes, int plane_tiles, cudaStream_t st) {
    if (planes) {  // the PSF spectra: [bins][S][Cw] (plane_tiles = S rows per bin)
        OutPlanes o{{planes[0], planes[1], planes[2], planes[3]}, plane_tiles, ldc};
        return p.F == 64 ? run_r2c<64>(src, nch, ldc, ntile, o, st) : run_r2c<32>(src, nch, ldc, ntile, o, st);
    }
    OutC64 o{c64, ntile, ldc};
    return p.F == 64 ? run_r2c<64>(src, nch, ldc, ntile, o, st) : run_r2c<32>(src, nch, ldc, ntile, o, st);
}

// the columns' spectra for the tensor-core contraction: grouped planes
// (ldc a multiple of 8)
template <class Src>
cudaError_t r2c_grouped(const FftPlan& p, Src src, int nch, int ldc, int ntile,
                        __nv_bfloat16* const* planes, int ncolp, cudaStream_t st) {
    OutPlanesG o{{planes[0], planes[1], planes[2], planes[3]}, ncolp, p.bins};
    return p.F == 64 ? run_r2c<64>(src, nch, ldc, ntile, o, st) : run_r2c<32>(src, nch, ldc, ntile, o, st);
}

template <int F, int LAYOUT, class Dst>
cudaError_t run_c2r_l(const float2* in, int nch, int ldc, int ntile, int off, int B, Dst dst,
                      cudaStream_t st) {
    if (ldc % 8 != 0) return cudaErrorInvalidValue;  // whole 8-channel groups per row
    const size_t smem = fft_smem<F>(false);
    cudaError_t e = cudaFuncSetAttribute(k_fft_c2r<F, Dst, LAYOUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)ntile, (unsigned)((nch + FftSize<F>::C2R_CH - 1) / FftSize<F>::C2R_CH));
    k_fft_c2r<F, Dst, LAYOUT><<<grid, FftSize<F>::C2R_THREADS, smem, st>>>(in, nch, ldc, ntile, off, B,
                                                                             1.0f / (F * F), dst);
    count_launch();
    return cudaGetLastError();
}
// tc: the spectra come group-major from the tensor-core contraction (the
// forward's columns outer, the adjoint's bins outer), else complex64 from the
// CUDA-core contraction
template <int F, class Dst>
cudaError_t run_c2r(bool tc, bool adjoint, const float2* in, int nch, int ldc, int ntile, int off, int B,
                    Dst dst, cudaStream_t st) {
    if (!tc) return run_c2r_l<F, 0>(in, nch, ldc, ntile, off, B, dst, st);
    return adjoint ? run_c2r_l<F, 2>(in, nch, ldc, ntile, off, B, dst, st)
                   : run_c2r_l<F, 1>(in, nch, ldc, ntile, off, B, dst, st);
}

}  // namespace

// ------------------------------------------------------------------ plan --
bool fft_plan_for(const Geo& g, FftPlan* p, int force_F, int frames, int tc_products) {
    FftPlan best{};
    double best_t = 1e300;
    for (int F : {32, 64}) {
        if (force_F && F != force_F) continue;
        const int B = F - 2 * g.h;
        if (B < 4) continue;
        FftPlan q{};
        q.F = F;
        q.B = B;
        q.h = g.h;
        q.tiles_y = (g.Ly + B - 1) / B;
        q.tiles_x = (g.Lx + B - 1) / B;
        q.ntile = q.tiles_y * q.tiles_x;
        if (q.ntile > 64) continue;
        if (g.S > 256) continue;  // one thread per phase in the FP32 forward contraction
        q.bins = F * (F / 2 + 1);
        q.Cf = (g.C + 7) & ~7;
        q.Sf = (g.S + 7) & ~7;
        // BF16 plane rows in whole 256-byte blocks: the contractions' PSF tiles
        // (64 or 128 channels of a row) then never share an L2 line with their
        // neighbours
        q.Cw = (g.C + 127) & ~127;
        q.Sw = (g.S + 7) & ~7;
        // complex64, split BF16 (4 planes) or BF16 (2 planes)
        const double spectra = (double)q.bins * g.S * q.Cf * (tc_products == 2 ? 4.0 : 8.0);
        if (spectra > 96e9) continue;  // keep the cached spectra well inside HBM
        // complex multiply-adds at 8 flops: FP32 FMA on the CUDA cores, or two
        // or three BF16 tensor-core products per term
        const double flops = (double)q.bins * g.S * q.ntile * frames * g.C * 8.0;
        const double rate = tc_products ? 1.7e15 / tc_products : 6.0e13;
        // transforms: one F x F patch per tile, frame and channel
        const double xform = (double)q.ntile * frames * (g.C + g.S) * 2.0 * F * F * 8.0;
        // the tensor-core contraction streams the spectra once per 64 columns
        const double passes = tc_products ? (double)((q.ntile * frames + 63) / 64) : 1.0;
        const double t = std::max(spectra * passes / 6.0e12, flops / rate) + xform / 4.0e12;
        if (t < best_t) {
            best_t = t;
            best = q;
        }
    }
    if (best.F == 0) return false;
    *p = best;
    return true;
}

// -------------------------------------------------------------- launchers --
cudaError_t fft_init(const FftPlan& p, const Geo& g, const float* W32, const FftBuffers& b,
                     cudaStream_t st) {
    cudaError_t e = upload_twiddles();
    if (e != cudaSuccess) return e;
    TapSrc src{W32, g.T, g.Spad, g.Cpad};
    // "tiles" = phases s, channels = c: Wf[bin][s][c]
    if (b.Wp[0]) return r2c_any(p, src, g.C, p.Cw, g.S, nullptr, b.Wp, g.S, st);
    return r2c_any(p, src, g.C, p.Cf, g.S, b.Wf, nullptr, 0, st);
}

cudaError_t fft_forward(const FftPlan& p, const Geo& g, const FftBuffers& b, int nf, const float* vcm,
                        float* img_out, float* rcm, const float* ycm, float* rimg, float eps,
                        cudaStream_t st, cudaEvent_t* ev) {
    const int64_t L2 = (int64_t)g.Ly * g.Lx;
    const int ncol = nf * p.ntile;
    ImgSrc src{vcm, g.Ly, g.Lx, p.h, p.B, p.tiles_x, p.ntile, (int64_t)g.C * L2};
    cudaError_t e = b.cg ? r2c_grouped(p, src, g.C, p.Cw, ncol, b.Xp, b.ncolp, st)
                         : r2c_any(p, src, g.C, p.Cf, ncol, b.Xh, nullptr, 0, st);
    if (e != cudaSuccess) return e;
    if (ev && (e = cudaEventRecord(ev[0], st)) != cudaSuccess) return e;
    e = b.cg ? cgemm_forward(b.cg, ncol, st) : contract_fwd_all(p, g, b.Wf, b.Xh, b.Yh, ncol, st);
    if (e != cudaSuccess) return e;
    if (ev && (e = cudaEventRecord(ev[1], st)) != cudaSuccess) return e;
    HvDst dst{img_out, rcm, ycm, rimg, eps, g.N, g.W, g.Ly, g.Lx, p.B, p.tiles_x, p.ntile,
              (int64_t)g.S * L2, (int64_t)g.H * g.W};
    return p.F == 64 ? run_c2r<64>(b.cg != nullptr, false, b.Yh, g.S, p.Sf, ncol, 2 * p.h, p.B, dst, st)
                     : run_c2r<32>(b.cg != nullptr, false, b.Yh, g.S, p.Sf, ncol, 2 * p.h, p.B, dst, st);
}

cudaError_t fft_backward(const FftPlan& p, const Geo& g, const FftBuffers& b, int nf, const float* rcm,
                         float* xcm, float* stack_out, cudaStream_t st, cudaEvent_t* ev) {
    const int64_t L2 = (int64_t)g.Ly * g.Lx;
    const int ncol = nf * p.ntile;
    ImgSrc src{rcm, g.Ly, g.Lx, p.h, p.B, p.tiles_x, p.ntile, (int64_t)g.S * L2};
    cudaError_t e = b.cg ? r2c_grouped(p, src, g.S, p.Sw, ncol, b.Yp, b.ncolp, st)
                         : r2c_any(p, src, g.S, p.Sf, ncol, b.Yh, nullptr, 0, st);
    if (e != cudaSuccess) return e;
    if (ev && (e = cudaEventRecord(ev[0], st)) != cudaSuccess) return e;
    e = b.cg ? cgemm_adjoint(b.cg, ncol, st) : contract_adj_all(p, g, b.Wf, b.Yh, b.Xh, ncol, st);
    if (e != cudaSuccess) return e;
    if (ev && (e = cudaEventRecord(ev[1], st)) != cudaSuccess) return e;
    VolDst dst{xcm, stack_out, g.N, g.S, g.H, g.W, g.Ly, g.Lx, p.B, p.tiles_x, p.ntile,
               (int64_t)g.C * L2, (int64_t)g.Nz * g.H * g.W};
    return p.F == 64 ? run_c2r<64>(b.cg != nullptr, true, b.Xh, g.C, p.Cf, ncol, 0, p.B, dst, st)
                     : run_c2r<32>(b.cg != nullptr, true, b.Xh, g.C, p.Cf, ncol, 0, p.B, dst, st);
}

static cudaError_t cm_copy(bool to, const float* src, const Geo& g, int planes, float* dst, cudaStream_t st) {
    const size_t smem = sizeof(float) * (size_t)g.W;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(to ? k_to_cm : k_from_cm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((unsigned)g.H, (unsigned)planes);
    if (to)
        k_to_cm<<<grid, 256, smem, st>>>(src, g, dst);
    else
        k_from_cm<<<grid, 256, smem, st>>>(src, g, dst);
    count_launch();
    return cudaGetLastError();
}
cudaError_t launch_poly_volume_cm(const float* v, const Geo& g, float* vcm, cudaStream_t st) {
    return cm_copy(true, v, g, g.Nz, vcm, st);
}
cudaError_t launch_depoly_volume_cm(const float* vcm, const Geo& g, float* v, cudaStream_t st) {
    return cm_copy(false, vcm, g, g.Nz, v, st);
}
cudaError_t launch_poly_image_cm(const float* y, const Geo& g, float* ycm, cudaStream_t st) {
    return cm_copy(true, y, g, 1, ycm, st);
}
cudaError_t launch_fill_cm(float* p, int64_t n, float val, cudaStream_t st) {
    k_fill_cm<<<grid_for(n), 256, 0, st>>>(p, n, val);
    count_launch();
    return cudaGetLastError();
}
cudaError_t launch_inv_cm(const float* x, int64_t n, float* inv, cudaStream_t st) {
    k_inv_cm<<<grid_for(n), 256, 0, st>>>(x, n, inv);
    count_launch();
    return cudaGetLastError();
}
cudaError_t launch_exact_bwd(const int64_t* list, int64_t n, int nf, const float* rimg,
                             const float* psf, const Geo& g, float* xcm, cudaStream_t st) {
    if (n <= 0 || nf <= 0) return cudaSuccess;
    int64_t blocks = (n * nf * 32 + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    k_exact_bwd<<<(unsigned)blocks, 256, 0, st>>>(list, n, nf, rimg, psf, g, xcm);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_exact_bwd_dev(const int* list, const int* n, const float* rimg, const float* psf,
                                 const Geo& g, float* xcm, cudaStream_t st) {
    k_exact_bwd_dev<<<152 * 8, 256, 0, st>>>(list, n, rimg, psf, g, xcm);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_low_list(const float* x, int64_t n, float frac, unsigned* mx, int* list, int* count,
                            cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(mx, 0, sizeof(unsigned), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(count, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    k_max_nonneg<<<grid_for(n), 256, 0, st>>>(x, n, mx);
    k_low_list<<<grid_for(n), 256, 0, st>>>(x, n, mx, frac, list, count);
    count_launch(2);
    return cudaGetLastError();
}

cudaError_t fft_forward_tab(const FftPlan& p, const Geo& g, const FftBuffers& b, const FrameCols* fr,
                            const int* colf, int col0, int ncol, float eps, cudaStream_t st) {
    TabSrc src{fr, colf, col0, p.h, p.B, true};
    cudaError_t e = b.cg ? r2c_grouped(p, src, g.C, p.Cw, ncol, b.Xp, b.ncolp, st)
                         : r2c_any(p, src, g.C, p.Cf, ncol, b.Xh, nullptr, 0, st);
    if (e != cudaSuccess) return e;
    e = b.cg ? cgemm_forward(b.cg, ncol, st) : contract_fwd_all(p, g, b.Wf, b.Xh, b.Yh, ncol, st);
    if (e != cudaSuccess) return e;
    TabHvDst dst{fr, colf, col0, g.N, p.B, eps};
    return p.F == 64 ? run_c2r<64>(b.cg != nullptr, false, b.Yh, g.S, p.Sf, ncol, 2 * p.h, p.B, dst, st)
                     : run_c2r<32>(b.cg != nullptr, false, b.Yh, g.S, p.Sf, ncol, 2 * p.h, p.B, dst, st);
}

cudaError_t fft_backward_tab(const FftPlan& p, const Geo& g, const FftBuffers& b, const FrameCols* fr,
                             const int* colf, int col0, int ncol, cudaStream_t st) {
    TabSrc src{fr, colf, col0, p.h, p.B, false};
    cudaError_t e = b.cg ? r2c_grouped(p, src, g.S, p.Sw, ncol, b.Yp, b.ncolp, st)
                         : r2c_any(p, src, g.S, p.Sf, ncol, b.Yh, nullptr, 0, st);
    if (e != cudaSuccess) return e;
    e = b.cg ? cgemm_adjoint(b.cg, ncol, st) : contract_adj_all(p, g, b.Wf, b.Yh, b.Xh, ncol, st);
    if (e != cudaSuccess) return e;
    TabVolDst dst{fr, colf, col0, g.N, g.S, p.B};
    return p.F == 64 ? run_c2r<64>(b.cg != nullptr, true, b.Xh, g.C, p.Cf, ncol, 0, p.B, dst, st)
                     : run_c2r<32>(b.cg != nullptr, true, b.Xh, g.C, p.Cf, ncol, 0, p.B, dst, st);
}

// one item per thread (no grid-stride tail), one flux partial per block
int update_cm_blocks(const Geo& g) { return (int)(((int64_t)g.S * g.Ly * g.Lx + 255) / 256); }
cudaError_t launch_update_cm(const float* vin, float* vout, const float* x, const float* inv,
                             const Geo& g, int nf, float* mip, double* flux_part, cudaStream_t st) {
    dim3 grid((unsigned)update_cm_blocks(g), (unsigned)nf);
    k_update_cm<<<grid, 256, 0, st>>>(vin, vout, x, inv, g, mip, flux_part);
    count_launch();
    return cudaGetLastError();
}

}  // namespace lfd
