// FP32 implicit-GEMM projections on the CUDA cores (FFMA): the plain FP32 GPU
// path that the tensor-core path is measured against.
//
//   forward   out[m][s]      = sum_D sum_c  Vp[m_base + m - off(D)][c] * Wp[D][s][c]
//   backward  out[m][(z,t)]  = sum_D sum_s  Rp[m_base + m + off(D)][s] * Wp[D][s][(z,t)]
//   off(D) = Dy*Lp + Dx  (padded lenslet-grid row offset, see lfd_internal.h)
//
// 128x128 output tile per 256-thread block, 8x8 outputs per thread, K staged
// through shared memory 16 at a time with register double buffering. Taps are
// split across blockIdx.z into separate partial outputs (summed later in a
// fixed order). Each thread sums one tap's K range in a fresh accumulator and
// adds it to the running total, which keeps FP32 rounding growth with the
// contraction length (up to ~7e6 terms) small.
#include "lfd_internal.h"

namespace lfd {
namespace {

constexpr int BM = 128, BN = 128, BK = 16;

template <bool FWD>
__global__ void __launch_bounds__(256, 1)
k_simt_conv(const float* __restrict__ A, const float* __restrict__ Wt, Geo g, int taps_per_split,
            float* __restrict__ out) {
    __shared__ __align__(16) float As[2][BK][BM];
    __shared__ __align__(16) float Bs[2][BK][BN];

    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int64_t m0 = (int64_t)blockIdx.x * BM;
    const int n0 = blockIdx.y * BN;
    const int split = blockIdx.z;
    const int T2 = g.T * g.T;
    const int tap_lo = split * taps_per_split;
    const int tap_hi = min(tap_lo + taps_per_split, T2);
    if (tap_lo >= tap_hi) return;  // uniform per block
    const int Kt = FWD ? g.Cpad : g.Spad;  // contraction length per tap
    const int lda = Kt;
    const int Nn = FWD ? g.Spad : g.Cpad;  // output width
    const int nk = Kt / BK;
    const int iters = (tap_hi - tap_lo) * nk;

    float acc[8][8], tot[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = tot[i][j] = 0.f;

    float4 ra[2], rb[2];
    auto load = [&](int it) {
        const int tap = tap_lo + it / nk;
        const int k0 = (it % nk) * BK;
        const int Dy = tap / g.T - g.h, Dx = tap % g.T - g.h;
        const int64_t off = (int64_t)Dy * g.Lp + Dx;
        const int64_t rbase = g.m_base + m0 + (FWD ? -off : off);
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const int idx = tid + p * 256;
            const int r = idx >> 2, q = idx & 3;
            ra[p] = *reinterpret_cast<const float4*>(A + (rbase + r) * lda + k0 + q * 4);
            if (FWD) {
                const int n = n0 + r;
                rb[p] = n < g.Spad
                            ? *reinterpret_cast<const float4*>(
                                  Wt + ((int64_t)tap * g.Spad + n) * g.Cpad + k0 + q * 4)
                            : make_float4(0.f, 0.f, 0.f, 0.f);
            } else {
                const int kk = idx >> 5, nq = idx & 31;
                const int n = n0 + nq * 4;
                rb[p] = n < g.Cpad
                            ? *reinterpret_cast<const float4*>(
                                  Wt + ((int64_t)tap * g.Spad + k0 + kk) * g.Cpad + n)
                            : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const int idx = tid + p * 256;
            const int r = idx >> 2, q = idx & 3;
            As[buf][q * 4 + 0][r] = ra[p].x;
            As[buf][q * 4 + 1][r] = ra[p].y;
            As[buf][q * 4 + 2][r] = ra[p].z;
            As[buf][q * 4 + 3][r] = ra[p].w;
            if (FWD) {
                Bs[buf][q * 4 + 0][r] = rb[p].x;
                Bs[buf][q * 4 + 1][r] = rb[p].y;
                Bs[buf][q * 4 + 2][r] = rb[p].z;
                Bs[buf][q * 4 + 3][r] = rb[p].w;
            } else {
                const int kk = idx >> 5, nq = idx & 31;
                *reinterpret_cast<float4*>(&Bs[buf][kk][nq * 4]) = rb[p];
            }
        }
    };

    load(0);
    store(0);
    __syncthreads();
    for (int it = 0; it < iters; ++it) {
        const int buf = it & 1;
        if (it + 1 < iters) load(it + 1);
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + ty * 4]);
            const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 + tx * 4]);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        if ((it + 1) % nk == 0) {  // end of a tap: fold into the running total
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    tot[i][j] += acc[i][j];
                    acc[i][j] = 0.f;
                }
        }
        if (it + 1 < iters) store(buf ^ 1);
        __syncthreads();
    }

    float* o = out + (int64_t)split * g.M_pad * Nn;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t m = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
#pragma unroll
        for (int hj = 0; hj < 2; ++hj) {
            const int n = n0 + hj * 64 + tx * 4;
            if (n < Nn)
                *reinterpret_cast<float4*>(o + m * Nn + n) =
                    make_float4(tot[i][hj * 4 + 0], tot[i][hj * 4 + 1], tot[i][hj * 4 + 2],
                                tot[i][hj * 4 + 3]);
        }
    }
}

int pick_splits(int64_t tiles, int T2, int sm_count) {
    // enough blocks for ~2 waves of one block per SM, never more than the taps
    int64_t want = (2LL * sm_count + tiles - 1) / tiles;
    if (want < 1) want = 1;
    if (want > T2) want = T2;
    // normalise so that every split gets at least one tap
    const int64_t tps = (T2 + want - 1) / want;
    return (int)((T2 + tps - 1) / tps);
}

}  // namespace

int simt_fwd_splits(const Geo& g, int sm_count) {
    const int64_t tiles = (g.M_pad / BM) * ((g.Spad + BN - 1) / BN);
    return pick_splits(tiles, g.T * g.T, sm_count);
}

int simt_bwd_splits(const Geo& g, int sm_count) {
    const int64_t tiles = (g.M_pad / BM) * ((g.Cpad + BN - 1) / BN);
    return pick_splits(tiles, g.T * g.T, sm_count);
}

cudaError_t launch_simt_forward(const float* vp32, const float* W32, const Geo& g, int nsplit,
                                float* out, cudaStream_t st) {
    const int T2 = g.T * g.T;
    const int tps = (T2 + nsplit - 1) / nsplit;
    dim3 grid((unsigned)(g.M_pad / BM), (unsigned)((g.Spad + BN - 1) / BN), (unsigned)nsplit);
    k_simt_conv<true><<<grid, 256, 0, st>>>(vp32, W32, g, tps, out);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_simt_backward(const float* rp32, const float* W32, const Geo& g, int nsplit,
                                 float* out, cudaStream_t st) {
    const int T2 = g.T * g.T;
    const int tps = (T2 + nsplit - 1) / nsplit;
    dim3 grid((unsigned)(g.M_pad / BM), (unsigned)((g.Cpad + BN - 1) / BN), (unsigned)nsplit);
    k_simt_conv<false><<<grid, 256, 0, st>>>(rp32, W32, g, tps, out);
    count_launch();
    return cudaGetLastError();
}

}  // namespace lfd
