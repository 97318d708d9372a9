// Layout kernels: PSF polyphase repack, volume / image (de)polyphase copies,
// and the forward-projection finishing passes (split reduction + ratio).
#include "lfd_internal.h"

namespace lfd {

std::atomic<uint64_t> g_launches{0};
std::atomic<int> g_fail_allocs{0};

namespace {

__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16* hi, __nv_bfloat16* lo, int64_t e) {
    __nv_bfloat16 h = __float2bfloat16_rn(x);
    hi[e] = h;
    if (lo) lo[e] = __float2bfloat16_rn(x - __bfloat162float(h));
}

inline int grid_for(int64_t n, int block = 256, int cap = 152 * 32) {
    int64_t b = (n + block - 1) / block;
    if (b < 1) b = 1;
    return (int)(b < cap ? b : cap);
}

// Wp[d][s][c] with d = (Dy+h)*T + (Dx+h), s = sy*N + sx, c = z*S + ty*N + tx:
// K[z][ty][tx][N*Dy + sy - ty + c0][N*Dx + sx - tx + c0], 0 outside [0,P).
__global__ void k_repack_psf(const float* __restrict__ psf, Geo g, float* __restrict__ W32,
                             __nv_bfloat16* __restrict__ whi, __nv_bfloat16* __restrict__ wlo) {
    const int64_t total = g.taps() * g.Spad * (int64_t)g.Cpad;
    const int c0 = (g.P - 1) / 2;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e % g.Cpad);
        const int64_t r = e / g.Cpad;
        const int s = (int)(r % g.Spad);
        const int d = (int)(r / g.Spad);
        float val = 0.f;
        if (c < g.C && s < g.S) {
            const int z = c / g.S, t = c % g.S;
            const int ty = t / g.N, tx = t % g.N, sy = s / g.N, sx = s % g.N;
            const int Dy = d / g.T - g.h, Dx = d % g.T - g.h;
            const int mi = g.N * Dy + sy - ty + c0, mj = g.N * Dx + sx - tx + c0;
            if (mi >= 0 && mi < g.P && mj >= 0 && mj < g.P)
                val = psf[((((int64_t)z * g.N + ty) * g.N + tx) * g.P + mi) * g.P + mj];
        }
        W32[e] = val;
        if (whi) split_bf16(val, whi, wlo, e);
    }
}

// v[z][Iy*N+ty][Ix*N+tx] -> vp[m_base + Iy*Lp + Ix][z*S + ty*N + tx]
__global__ void k_poly_volume(const float* __restrict__ v, Geo g, float* __restrict__ vp,
                              __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo) {
    const int64_t total = (int64_t)g.Ly * g.Lx * g.C;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e % g.C);
        const int64_t l = e / g.C;
        const int Iy = (int)(l / g.Lx), Ix = (int)(l % g.Lx);
        const int z = c / g.S, t = c % g.S, ty = t / g.N, tx = t % g.N;
        const float x = v[((int64_t)z * g.H + (int64_t)Iy * g.N + ty) * g.W + (int64_t)Ix * g.N + tx];
        const int64_t d = (g.m_base + (int64_t)Iy * g.Lp + Ix) * g.Cpad + c;
        vp[d] = x;
        if (hi) split_bf16(x, hi, lo, d);
    }
}

// inverse of k_poly_volume, from rows row0 + Iy*Lp + Ix
__global__ void k_depoly_volume(const float* __restrict__ vp, int64_t row0, Geo g,
                                float* __restrict__ v) {
    const int64_t total = (int64_t)g.Nz * g.H * g.W;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e % g.W);
        const int64_t zi = e / g.W;
        const int i = (int)(zi % g.H), z = (int)(zi / g.H);
        const int Iy = i / g.N, ty = i % g.N, Ix = j / g.N, tx = j % g.N;
        const int c = z * g.S + ty * g.N + tx;
        v[e] = vp[(row0 + (int64_t)Iy * g.Lp + Ix) * g.Cpad + c];
    }
}

// sum of split partials [split][M_pad][Cpad] -> v[Nz][H][W]
__global__ void k_sum_depoly_volume(const float* __restrict__ parts, int nsplit, Geo g,
                                    float* __restrict__ v) {
    const int64_t total = (int64_t)g.Nz * g.H * g.W;
    const int64_t stride = g.M_pad * g.Cpad;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e % g.W);
        const int64_t zi = e / g.W;
        const int i = (int)(zi % g.H), z = (int)(zi / g.H);
        const int Iy = i / g.N, ty = i % g.N, Ix = j / g.N, tx = j % g.N;
        const int64_t o = ((int64_t)Iy * g.Lp + Ix) * g.Cpad + z * g.S + ty * g.N + tx;
        float s = 0.f;
        for (int q = 0; q < nsplit; ++q) s += parts[o + q * stride];
        v[e] = s;
    }
}

// y[Iy*N+sy][Ix*N+sx] -> dst[row0 + Iy*Lp + Ix][sy*N + sx]
__global__ void k_poly_image(const float* __restrict__ y, Geo g, float* __restrict__ dst,
                             int64_t row0, __nv_bfloat16* __restrict__ hi,
                             __nv_bfloat16* __restrict__ lo) {
    const int64_t total = (int64_t)g.H * g.W;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e % g.W), i = (int)(e / g.W);
        const int Iy = i / g.N, sy = i % g.N, Ix = j / g.N, sx = j % g.N;
        const int64_t d = (row0 + (int64_t)Iy * g.Lp + Ix) * g.Spad + sy * g.N + sx;
        dst[d] = y[e];
        if (hi) split_bf16(y[e], hi, lo, d);
    }
}

// sum of forward partials [split][M_pad][Spad] -> y_out[H][W]
__global__ void k_fwd_finish_image(const float* __restrict__ parts, int nsplit, Geo g,
                                   float* __restrict__ y) {
    const int64_t total = (int64_t)g.H * g.W;
    const int64_t stride = g.M_pad * g.Spad;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e % g.W), i = (int)(e / g.W);
        const int Iy = i / g.N, sy = i % g.N, Ix = j / g.N, sx = j % g.N;
        const int64_t o = ((int64_t)Iy * g.Lp + Ix) * g.Spad + sy * g.N + sx;
        float s = 0.f;
        for (int q = 0; q < nsplit; ++q) s += parts[o + q * stride];
        y[e] = s;
    }
}

// r = y / (Hv + eps) (0 where Hv + eps <= 0), written to the padded image
// buffer the backprojection reads; Hv = sum of the split partials.
__global__ void k_fwd_finish_ratio(const float* __restrict__ parts, int nsplit,
                                   const float* __restrict__ ypoly, float eps, Geo g,
                                   float* __restrict__ rp, __nv_bfloat16* __restrict__ hi,
                                   __nv_bfloat16* __restrict__ lo) {
    const int64_t total = (int64_t)g.Ly * g.Lx * g.S;
    const int64_t stride = g.M_pad * g.Spad;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int s = (int)(e % g.S);
        const int64_t l = e / g.S;
        const int Iy = (int)(l / g.Lx), Ix = (int)(l % g.Lx);
        const int64_t o = ((int64_t)Iy * g.Lp + Ix) * g.Spad + s;
        float hv = 0.f;
        for (int q = 0; q < nsplit; ++q) hv += parts[o + q * stride];
        const float den = hv + eps;
        const float r = den > 0.f ? ypoly[o] / den : 0.f;
        const int64_t d = g.m_base * g.Spad + o;
        rp[d] = r;
        if (hi) split_bf16(r, hi, lo, d);
    }
}

// 1 / (H^T 1) from the split partials of the backprojection of ones; 0 where
// H^T 1 <= 0.
__global__ void k_inv_ht1(const float* __restrict__ parts, int nsplit, Geo g,
                          float* __restrict__ inv) {
    const int64_t total = (int64_t)g.Ly * g.Lx * g.C;
    const int64_t stride = g.M_pad * g.Cpad;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e % g.C);
        const int64_t l = e / g.C;
        const int64_t o = ((l / g.Lx) * g.Lp + (l % g.Lx)) * g.Cpad + c;
        float s = 0.f;
        for (int q = 0; q < nsplit; ++q) s += parts[o + q * stride];
        inv[o] = s > 0.f ? 1.0f / s : 0.f;
    }
}

__global__ void k_fill(float* __restrict__ p, int64_t n, float val) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x)
        p[e] = val;
}

}  // namespace

cudaError_t launch_fill(float* p, int64_t n, float val, cudaStream_t st) {
    k_fill<<<grid_for(n), 256, 0, st>>>(p, n, val);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_repack_psf(const float* psf, const Geo& g, float* W32, __nv_bfloat16* whi,
                              __nv_bfloat16* wlo, cudaStream_t st) {
    k_repack_psf<<<grid_for(g.taps() * g.Spad * (int64_t)g.Cpad), 256, 0, st>>>(psf, g, W32, whi, wlo);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_poly_volume(const float* v, const Geo& g, float* vp32, __nv_bfloat16* hi,
                               __nv_bfloat16* lo, cudaStream_t st) {
    k_poly_volume<<<grid_for((int64_t)g.Ly * g.Lx * g.C), 256, 0, st>>>(v, g, vp32, hi, lo);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_depoly_volume(const float* vp32, int64_t row0, const Geo& g, float* v,
                                 cudaStream_t st) {
    k_depoly_volume<<<grid_for((int64_t)g.Nz * g.H * g.W), 256, 0, st>>>(vp32, row0, g, v);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_sum_depoly_volume(const float* parts, int nsplit, const Geo& g, float* v,
                                     cudaStream_t st) {
    k_sum_depoly_volume<<<grid_for((int64_t)g.Nz * g.H * g.W), 256, 0, st>>>(parts, nsplit, g, v);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_poly_image(const float* y, const Geo& g, float* dst, int64_t row0,
                              __nv_bfloat16* hi, __nv_bfloat16* lo, cudaStream_t st) {
    k_poly_image<<<grid_for((int64_t)g.H * g.W), 256, 0, st>>>(y, g, dst, row0, hi, lo);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_fwd_finish_image(const float* parts, int nsplit, const Geo& g, float* y_out,
                                    cudaStream_t st) {
    k_fwd_finish_image<<<grid_for((int64_t)g.H * g.W), 256, 0, st>>>(parts, nsplit, g, y_out);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_fwd_finish_ratio(const float* parts, int nsplit, const float* ypoly, float eps,
                                    const Geo& g, float* rp32, __nv_bfloat16* hi,
                                    __nv_bfloat16* lo, cudaStream_t st) {
    k_fwd_finish_ratio<<<grid_for((int64_t)g.Ly * g.Lx * g.S), 256, 0, st>>>(
        parts, nsplit, ypoly, eps, g, rp32, hi, lo);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_inv_ht1(const float* parts, int nsplit, const Geo& g, float* inv,
                           cudaStream_t st) {
    k_inv_ht1<<<grid_for((int64_t)g.Ly * g.Lx * g.C), 256, 0, st>>>(parts, nsplit, g, inv);
    count_launch();
    return cudaGetLastError();
}

}  // namespace lfd
