// Fused RL update (multiplicative step, clamp, z-MIP, flux) and the
// DCT-entropy metric of Section 2.2.
#include <algorithm>

#include "lfd_internal.h"

namespace lfd {
namespace {

__device__ __forceinline__ double warp_sum(double x) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// block-wide sum in a fixed order (deterministic); all threads get the result
__device__ double block_sum(double x, double* red) {
    x = warp_sum(x);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) red[w] = x;
    __syncthreads();
    double t = 0.0;
    for (int i = 0; i < nw; ++i) t += red[i];
    __syncthreads();
    return t;
}

// One block per lenslet (Iy, Ix); thread t < S walks the depths of phase t.
//   v_new = v * x * inv   (x = H^T r, inv = 1 / H^T 1, 0 where H^T 1 = 0)
//   v_new = max(0, v_new) with NaN -> 0
// and, on the fly, the z-maximum of v_new for pixel (Iy*N + ty, Ix*N + tx)
// and this lenslet's share of the flux sum(H^T1 * v_new) = sum(v * x) taken
// where H^T 1 > 0: compensated FP32 over a thread's depths, FP64 across
// threads (FP64 arithmetic per voxel would bound the kernel on the GB300's
// FP64 rate).
__global__ void __launch_bounds__(256) k_update(
    const float* __restrict__ vin, float* __restrict__ vout, __nv_bfloat16* __restrict__ hi,
    __nv_bfloat16* __restrict__ lo, const float* __restrict__ parts, int nsplit,
    const float* __restrict__ inv, Geo g, float* __restrict__ mip, double* __restrict__ flux_part) {
    __shared__ double red[32];
    const int l = blockIdx.x;
    const int Iy = l / g.Lx, Ix = l % g.Lx;
    const int64_t m = (int64_t)Iy * g.Lp + Ix;
    const int64_t grow = (g.m_base + m) * g.Cpad;
    const int64_t orow = m * g.Cpad;
    const int64_t pstride = g.M_pad * g.Cpad;
    double flux = 0.0;
    for (int t = threadIdx.x; t < g.S; t += blockDim.x) {
        float mx = 0.f;
        float fs = 0.f, fc = 0.f;  // this thread's depths: compensated FP32 sum
#pragma unroll 4
        for (int z = 0; z < g.Nz; ++z) {
            const int c = z * g.S + t;
            float x = parts[orow + c];
            for (int q = 1; q < nsplit; ++q) x += parts[orow + c + q * pstride];
            const float iv = inv[orow + c];
            const float vo = vin[grow + c];
            float vn = 0.f;
            if (iv > 0.f) {
                const float vx = vo * x;
                vn = vx * iv;
                kahan_add(fs, fc, vx);
            }
            vn = vn > 0.f ? vn : 0.f;  // clamp; a NaN compares false and becomes 0
            vout[grow + c] = vn;
            if (hi) {
                const __nv_bfloat16 h = __float2bfloat16_rn(vn);
                hi[grow + c] = h;
                if (lo) lo[grow + c] = __float2bfloat16_rn(vn - __bfloat162float(h));
            }
            mx = fmaxf(mx, vn);
        }
        const int ty = t / g.N, tx = t % g.N;
        mip[((int64_t)Iy * g.N + ty) * g.W + (int64_t)Ix * g.N + tx] = mx;
        flux += (double)fs - (double)fc;
    }
    const double f = block_sum(flux, red);
    if (threadIdx.x == 0) flux_part[l] = f;
}

// z-maximum projection straight from a padded channels-last volume
__global__ void k_mip(const float* __restrict__ vp, Geo g, float* __restrict__ mip) {
    const int l = blockIdx.x;
    const int Iy = l / g.Lx, Ix = l % g.Lx;
    const int64_t grow = (g.m_base + (int64_t)Iy * g.Lp + Ix) * g.Cpad;
    for (int t = threadIdx.x; t < g.S; t += blockDim.x) {
        float mx = 0.f;
        for (int z = 0; z < g.Nz; ++z) mx = fmaxf(mx, vp[grow + z * g.S + t]);
        const int ty = t / g.N, tx = t % g.N;
        mip[((int64_t)Iy * g.N + ty) * g.W + (int64_t)Ix * g.N + tx] = mx;
    }
}

// z-maximum projection of a volume in stack order [Nz][H][W]
__global__ void k_mip_stack(const float* __restrict__ v, int Nz, int64_t HW, float* __restrict__ mip) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < HW;
         e += (int64_t)gridDim.x * blockDim.x) {
        float mx = 0.f;
        for (int z = 0; z < Nz; ++z) mx = fmaxf(mx, v[z * HW + e]);
        mip[e] = mx;
    }
}

// Row transform (Eq. 1 along the rows, basis of Eqs. 2-4 tabulated in
// cosW[u][x]) G[u][y] = sum_x f[y][x] C_u(x; W), u < XS (stored transposed,
// for the column transform), and the row energy rowE2[y] = sum_x f[y][x]^2
// (FP64). A block holds ROWS rows in shared memory (8, fewer for very wide
// images); warp w takes the basis rows u = w, w + 8, ... and applies each to
// all the block's rows (one basis load per ROWS products, ROWS independent
// sums per lane; the basis values of four steps are loaded together). The products and sums are double-float on the
// FP32 units: the basis is an FP64 value split as hi + lo, each product
// f * hi is kept exactly as p + e (FMA), and each running sum is a
// compensated pair, rounded to FP64 at the end (about 44 significant bits,
// without the slow FP64 pipe of this GPU).
template <int ROWS>
__global__ void __launch_bounds__(256) k_dct_rows(const float* __restrict__ f, const float2* __restrict__ cosW,
                                                  int H, int W, int XS, double* __restrict__ G,
                                                  double* __restrict__ rowE2) {
    extern __shared__ float rows[];  // [ROWS][W]
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int y0 = blockIdx.x * ROWS;
    const int nr = min(ROWS, H - y0);
    {  // frame blockIdx.y
        f += (int64_t)blockIdx.y * H * W;
        G += (int64_t)blockIdx.y * H * XS;
        rowE2 += (int64_t)blockIdx.y * H;
    }
    for (int r = w; r < ROWS; r += nw) {
        double e2 = 0.0;
        for (int x = lane; x < W; x += 32) {
            const float a = r < nr ? f[(int64_t)(y0 + r) * W + x] : 0.f;
            rows[r * W + x] = a;
            e2 += (double)a * (double)a;
        }
        e2 = warp_sum(e2);
        if (lane == 0 && r < nr) rowE2[y0 + r] = e2;
    }
    __syncthreads();
    for (int u = w; u < XS; u += nw) {
        const float2* cb = cosW + (int64_t)u * W;
        float sh[ROWS], sl[ROWS];
#pragma unroll
        for (int r = 0; r < ROWS; ++r) sh[r] = sl[r] = 0.f;
        // the basis values of the next four steps are loaded while the
        // current ones are used
        float2 c[4], cn[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) c[k] = lane + 32 * k < W ? cb[lane + 32 * k] : make_float2(0.f, 0.f);
        for (int x0 = lane; x0 < W; x0 += 128) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int xn = x0 + 128 + 32 * k;
                cn[k] = xn < W ? cb[xn] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int x = x0 + 32 * k;
                if (x >= W) break;
#pragma unroll
                for (int r = 0; r < ROWS; ++r) {
                    const float m = rows[r * W + x];
                    const float p = m * c[k].x;
                    const float e = fmaf(m, c[k].y, fmaf(m, c[k].x, -p));  // m*hi - p exactly, plus m*lo
                    const float t = sh[r] + p;                              // two-sum of sh + p
                    const float bp = t - sh[r];
                    sl[r] += ((sh[r] - (t - bp)) + (p - bp)) + e;
                    sh[r] = t;
                }
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) c[k] = cn[k];
        }
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
            const double s = warp_sum((double)sh[r] + (double)sl[r]);
            if (lane == 0 && r < nr) G[(int64_t)u * H + y0 + r] = s;
        }
    }
}
// Column transform coef[v][u] = sum_y C_v(y; H) G[u][y] (FP64) inside the
// triangular region; block (u, group of 8 rows v), one warp per v, four
// partial sums per lane.
__global__ void k_dct_cols(const double* __restrict__ G, const double* __restrict__ cosH, int H,
                           int XS, int YS, double* __restrict__ coef) {
    const int u = blockIdx.x;
    G += (int64_t)blockIdx.z * H * XS;  // frame blockIdx.z
    coef += (int64_t)blockIdx.z * XS * YS;
    const int lane = threadIdx.x & 31, v = blockIdx.y * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (v >= YS) return;
    const bool in = (int64_t)u * YS + (int64_t)v * XS < (int64_t)XS * YS;
    double s = 0.0;
    if (in) {
        const double* cb = cosH + (int64_t)v * H;
        const double* gu = G + (int64_t)u * H;
        double a[4] = {0.0, 0.0, 0.0, 0.0};
        for (int y0 = lane; y0 < H; y0 += 128) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int y = y0 + 32 * k;
                if (y < H) a[k] = fma(cb[y], gu[y], a[k]);
            }
        }
        s = warp_sum((a[0] + a[1]) + (a[2] + a[3]));
    }
    if (lane == 0) coef[(int64_t)v * XS + u] = in ? s : 0.0;
}

// E = -(1/G_S) sum_S |p| log2 |p|, p = F / ||F||_2 (Eqs. 5, 6, 12), and the
// flux total, in two kernels. With N = ||F||_2 and, over the region S,
// S1 = sum |F| log2 |F|, S2 = sum |F| (terms with F = 0 left out),
//   sum_S p log2 p = (S1 - log2(N) S2) / N,
// so the sums need no N and are split over kEntBlocks blocks per frame
// (each a fixed slice: N^2 over the region, or the row energies of the whole
// image; S1; S2; the flux partials), and one warp per frame adds the block
// sums in a fixed order. All FP64.
constexpr int kEntBlocks = 16;
__global__ void k_entropy_part(const double* __restrict__ coef, const double* __restrict__ rowE2, int H,
                               int XS, int YS, int l2_over_region, const double* __restrict__ flux_part,
                               int nflux, double* __restrict__ part) {
    __shared__ double red[32];
    const int fr = blockIdx.y, b = blockIdx.x, nb = gridDim.x;
    coef += (int64_t)fr * XS * YS;
    rowE2 += (int64_t)fr * H;
    if (flux_part) flux_part += (int64_t)fr * nflux;
    part += ((int64_t)fr * nb + b) * 4;
    const int n = XS * YS;
    const int i0 = (int)((int64_t)b * n / nb), i1 = (int)((int64_t)(b + 1) * n / nb);
    double a = 0.0, s1 = 0.0, s2 = 0.0;
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const int v = i / XS, u = i % XS;
        if ((int64_t)u * YS + (int64_t)v * XS < (int64_t)XS * YS) {
            const double c = fabs(coef[i]);
            if (l2_over_region) a += c * c;
            if (c > 0.0) {
                s1 += c * log2(c);
                s2 += c;
            }
        }
    }
    if (!l2_over_region) {
        const int y0 = (int)((int64_t)b * H / nb), y1 = (int)((int64_t)(b + 1) * H / nb);
        for (int y = y0 + threadIdx.x; y < y1; y += blockDim.x) a += rowE2[y];
    }
    double fl = 0.0;
    if (flux_part) {
        const int f0 = (int)((int64_t)b * nflux / nb), f1 = (int)((int64_t)(b + 1) * nflux / nb);
        for (int i = f0 + threadIdx.x; i < f1; i += blockDim.x) fl += flux_part[i];
    }
    a = block_sum(a, red);
    s1 = block_sum(s1, red);
    s2 = block_sum(s2, red);
    fl = block_sum(fl, red);
    if (threadIdx.x == 0) {
        part[0] = a;
        part[1] = s1;
        part[2] = s2;
        part[3] = fl;
    }
}

__global__ void k_entropy_fin(const double* __restrict__ part, int nb, int XS, int YS, int with_flux,
                              double* __restrict__ out_entropy, double* __restrict__ out_flux, int out_stride) {
    const int fr = blockIdx.x;
    part += (int64_t)fr * nb * 4;
    if (threadIdx.x != 0) return;
    double a = 0.0, s1 = 0.0, s2 = 0.0, fl = 0.0;
    for (int b = 0; b < nb; ++b) {
        a += part[4 * b];
        s1 += part[4 * b + 1];
        s2 += part[4 * b + 2];
        fl += part[4 * b + 3];
    }
    const double norm = sqrt(a);
    const double ent = norm > 0.0 ? (s1 - log2(norm) * s2) / norm : 0.0;
    out_entropy[(int64_t)fr * out_stride] = norm > 0.0 ? -ent / (0.5 * (double)XS * (double)YS) : 0.0;
    if (with_flux && out_flux) out_flux[(int64_t)fr * out_stride] = fl;
}

// r = y / (hv + eps) per pixel, 0 where hv + eps <= 0 (the ratio of an RL
// iteration whose forward projection was summed outside the library)
__global__ void k_ratio_image(const float* __restrict__ y, const float* __restrict__ hv, float eps,
                              int64_t n, float* __restrict__ r) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const float den = hv[e] + eps;
        r[e] = den > 0.f ? y[e] / den : 0.f;
    }
}

// out[0] = sum of p[0..n) in a fixed order (one block)
__global__ void k_sum_doubles(const double* __restrict__ p, int64_t n, double* __restrict__ out) {
    __shared__ double red[32];
    double a = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) a += p[i];
    a = block_sum(a, red);
    if (threadIdx.x == 0) out[0] = a;
}

}  // namespace

cudaError_t launch_ratio_image(const float* y, const float* hv, float eps, int64_t n, float* r,
                               cudaStream_t st) {
    int64_t b = (n + 255) / 256;
    k_ratio_image<<<(unsigned)(b < 4864 ? (b > 0 ? b : 1) : 4864), 256, 0, st>>>(y, hv, eps, n, r);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_sum_doubles(const double* p, int64_t n, double* out, cudaStream_t st) {
    k_sum_doubles<<<1, 256, 0, st>>>(p, n, out);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_update(const float* vin, float* vout, __nv_bfloat16* hi, __nv_bfloat16* lo,
                          const float* parts, int nsplit, const float* inv, const Geo& g,
                          float* mip, double* flux_part, cudaStream_t st) {
    const int threads = g.S >= 256 ? 256 : ((g.S + 31) / 32) * 32;
    k_update<<<g.Ly * g.Lx, threads, 0, st>>>(vin, vout, hi, lo, parts, nsplit, inv, g, mip,
                                              flux_part);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_mip(const float* vp32, const Geo& g, float* mip, cudaStream_t st) {
    const int threads = g.S >= 256 ? 256 : ((g.S + 31) / 32) * 32;
    k_mip<<<g.Ly * g.Lx, threads, 0, st>>>(vp32, g, mip);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_mip_stack(const float* v, int Nz, int64_t HW, float* mip, cudaStream_t st) {
    int64_t b = (HW + 255) / 256;
    k_mip_stack<<<(unsigned)(b < 4864 ? b : 4864), 256, 0, st>>>(v, Nz, HW, mip);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_metric(const float* mip, const float2* cosW, const double* cosH, int H, int W,
                          int XS, int YS, int l2_over_region, double* G, double* rowE2,
                          double* coef, const double* flux_part, int nflux, double* out_entropy,
                          double* out_flux, cudaStream_t st, int nf, int out_stride) {
    // 8 rows per block, fewer where 8 rows of floats exceed 200 KB of shared memory
    const size_t rowb = (size_t)W * sizeof(float);
    const int rows = rowb * 8 <= 200 * 1024 ? 8 : rowb * 4 <= 200 * 1024 ? 4 : rowb * 2 <= 200 * 1024 ? 2 : 1;
    const size_t smem = rows * rowb;
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    auto launch = [&](auto kern) -> cudaError_t {
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        kern<<<dim3((H + rows - 1) / rows, nf), 256, smem, st>>>(mip, cosW, H, W, XS, G, rowE2);
        return cudaSuccess;
    };
    cudaError_t e = rows == 8 ? launch(k_dct_rows<8>) : rows == 4 ? launch(k_dct_rows<4>)
                  : rows == 2 ? launch(k_dct_rows<2>) : launch(k_dct_rows<1>);
    if (e != cudaSuccess) return e;
    k_dct_cols<<<dim3(XS, (YS + 7) / 8, nf), 256, 0, st>>>(G, cosH, H, XS, YS, coef);
    // the entropy's block sums go to the scratch past the frames' coefficients
    static_assert(4 * kEntBlocks <= kMetricScratch, "entropy block sums exceed the metric scratch");
    double* part = coef + (int64_t)nf * XS * YS;
    k_entropy_part<<<dim3(kEntBlocks, nf), 256, 0, st>>>(coef, rowE2, H, XS, YS, l2_over_region, flux_part, nflux,
                                                         part);
    k_entropy_fin<<<nf, 32, 0, st>>>(part, kEntBlocks, XS, YS, flux_part != nullptr, out_entropy, out_flux,
                                     out_stride);
    count_launch(4);
    return cudaGetLastError();
}

}  // namespace lfd
