// DCT entropy of a z-maximum projection image with no memory allocation.
//
// Variant of the metric kernels (k_update.cu) for callers that cannot
// allocate device memory: the intermediate row transform and the region
// coefficients live in one file-scope __device__ array instead of buffers a
// context owns, and the cosine basis is evaluated in the kernels instead of
// being read from host-built tables. The caller passes the image and the
// output; nothing else is touched.
#include <cmath>
#include <cstdio>

#include "lfd_internal.h"

namespace {

constexpr int kQsMaxH = 4096;
constexpr int kQsMaxW = 4096;
constexpr int kQsMaxXS = 128;
constexpr int kQsMaxYS = 128;
// G[H][XS] row transform, rowE2[H] row energies, coef[YS][XS] coefficients
constexpr long long kQsDoubles =
    (long long)kQsMaxH * kQsMaxXS + kQsMaxH + (long long)kQsMaxXS * kQsMaxYS;

// Shared by every call on a device and kept until the process exits
// (about 4.2 MB per GPU that loads the library).
static __device__ __align__(256) double g_qs_scratch[kQsDoubles];

// orthonormal DCT-II basis C_k(x; Z) = c(k, Z) cos((2x+1) pi k / (2Z)) (Eqs. 2-4)
__device__ __forceinline__ double qs_basis(int k, int x, int Z) {
    const double c = k == 0 ? sqrt(1.0 / Z) : sqrt(2.0 / Z);
    return c * cospi((2.0 * x + 1.0) * (double)k / (2.0 * Z));
}

__device__ __forceinline__ double qs_warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ double qs_block_sum(double v, double* red) {
    v = qs_warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double t = 0.0;
    for (int i = 0; i < nw; ++i) t += red[i];
    __syncthreads();
    return t;
}

// one block per image row y: G[y][u] for u < XS and the row energy
__global__ void k_qs_rows(const float* __restrict__ f, int H, int W, int XS, double* __restrict__ s) {
    __shared__ float row[kQsMaxW];
    __shared__ double red[32];
    double* G = s;
    double* rowE2 = s + (long long)H * XS;
    const int y = blockIdx.x;
    double e2 = 0.0;
    for (int x = threadIdx.x; x < W; x += blockDim.x) {
        const float a = f[(long long)y * W + x];
        row[x] = a;
        e2 += (double)a * (double)a;
    }
    const double tot = qs_block_sum(e2, red);
    if (threadIdx.x == 0) rowE2[y] = tot;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int u = w; u < XS; u += nw) {
        double acc = 0.0;
        for (int x = lane; x < W; x += 32) acc += (double)row[x] * qs_basis(u, x, W);
        acc = qs_warp_sum(acc);
        if (lane == 0) G[(long long)y * XS + u] = acc;
    }
}

// one block per column frequency u: F(u, v) for v in the triangle (Eq. 6)
__global__ void k_qs_cols(int H, int XS, int YS, double* __restrict__ s) {
    const double* G = s;
    double* coef = s + (long long)H * XS + H;
    const int u = blockIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int v = w; v < YS; v += nw) {
        const bool in = (long long)u * YS + (long long)v * XS < (long long)XS * YS;
        double acc = 0.0;
        if (in) {
            for (int y = lane; y < H; y += 32) acc += qs_basis(v, y, H) * G[(long long)y * XS + u];
            acc = qs_warp_sum(acc);
        }
        if (lane == 0) coef[(long long)v * XS + u] = in ? acc : 0.0;
    }
}

// E = -(1/G_S) sum_S |p| log2 |p|, p = F / ||F||_2 (Eqs. 5, 6, 12)
__global__ void k_qs_entropy(int H, int XS, int YS, int l2_over_region, const double* __restrict__ s,
                             double* __restrict__ out) {
    __shared__ double red[32];
    const double* rowE2 = s + (long long)H * XS;
    const double* coef = rowE2 + H;
    const int n = XS * YS;
    double a = 0.0;
    if (l2_over_region) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) a += coef[i] * coef[i];
    } else {
        for (int i = threadIdx.x; i < H; i += blockDim.x) a += rowE2[i];
    }
    const double norm = sqrt(qs_block_sum(a, red));
    double e = 0.0;
    if (norm > 0.0) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const int v = i / XS, u = i % XS;
            if ((long long)u * YS + (long long)v * XS < (long long)XS * YS) {
                const double p = fabs(coef[i]) / norm;
                if (p > 0.0) e += p * log2(p);
            }
        }
    }
    const double ent = qs_block_sum(e, red);
    if (threadIdx.x == 0) out[0] = norm > 0.0 ? -ent / (0.5 * (double)XS * (double)YS) : 0.0;
}

// Device address of the scratch array on the current device. It is looked up
// on every call (cheap, allocates nothing), so a reloaded module after a
// device reset never leaves a stale address behind.
cudaError_t qs_scratch(double** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_qs_scratch);
    if (e != cudaSuccess) return e;
    *out = static_cast<double*>(p);
    return cudaSuccess;
}

// true when p is device (or managed) memory the kernels may dereference; a
// host address handed to them would fault or read the wrong memory
bool qs_device_ptr(const void* p) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();  // an unregistered host pointer may report an error here
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" lfd_status lfd_quality_mip_static(const float* mip, int H, int W, int XS, int YS,
                                             int l2_over_region, double* entropy,
                                             void* cuda_stream) {
    if (!mip || !entropy) {
        std::fprintf(stderr, "lfd_quality_mip_static: NULL image or output pointer\n");
        return LFD_EINVAL;
    }
    if (H < 1 || W < 1 || H > kQsMaxH || W > kQsMaxW) {
        std::fprintf(stderr,
                     "lfd_quality_mip_static: image %d x %d is outside 1..%d x 1..%d, the size of "
                     "the static scratch\n",
                     H, W, kQsMaxH, kQsMaxW);
        return LFD_EINVAL;
    }
    if (XS < 1 || YS < 1 || XS > W || YS > H || XS > kQsMaxXS || YS > kQsMaxYS) {
        std::fprintf(stderr,
                     "lfd_quality_mip_static: region %d x %d must lie in 1..min(W, %d) x "
                     "1..min(H, %d)\n",
                     XS, YS, kQsMaxXS, kQsMaxYS);
        return LFD_EINVAL;
    }
    if (!qs_device_ptr(mip) || !qs_device_ptr(entropy)) {
        std::fprintf(stderr,
                     "lfd_quality_mip_static: the image and the output must be device memory "
                     "(this entry point stages nothing)\n");
        return LFD_EINVAL;
    }
    double* s = nullptr;
    cudaError_t e = qs_scratch(&s);
    if (e != cudaSuccess) {
        std::fprintf(stderr, "lfd_quality_mip_static: cudaGetSymbolAddress: %s\n", cudaGetErrorString(e));
        return LFD_ECUDA;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    k_qs_rows<<<H, 256, 0, st>>>(mip, H, W, XS, s);
    k_qs_cols<<<XS, 256, 0, st>>>(H, XS, YS, s);
    k_qs_entropy<<<1, 256, 0, st>>>(H, XS, YS, l2_over_region, s, entropy);
    lfd::count_launch(3);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        std::fprintf(stderr, "lfd_quality_mip_static: launch: %s\n", cudaGetErrorString(e));
        return LFD_ECUDA;
    }
    return LFD_OK;
}
