// Internal declarations of liblfd: problem geometry, the context, kernel
// launchers. Not part of the public ABI (include/lfd.h is).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <map>
#include <string>
#include <vector>

#include "lfd.h"

namespace lfd {

// ---------------------------------------------------------------- geometry --
// Polyphase form of the light-field projection (the PSF repack of the
// forward model in include/lfd.h). Pixel i = Nnum*I + s (lenslet I, phase s),
// voxel i' = Nnum*I' + t. With D = I - I' the PSF index is
// m = Nnum*D + s - t + c, so
//   Hv[I][s]      = sum_D sum_{(z,t)} V[I-D][(z,t)] * Wp[D][s][(z,t)]
//   HtR[I'][(z,t)] = sum_D sum_s     R[I'+D][s]     * Wp[D][s][(z,t)]
// with Wp[D][s][(z,t)] = K[z][t][m_y][m_x] (0 outside the window). Every pair
// (s, t) has exactly k = P/Nnum valid D per axis; the union over pairs is
// D in [-h, h], h = (k+1)/2, i.e. T = k+2 taps per axis.
//
// Lenslet-grid buffers are flattened with a zero halo so that a tap shift is a
// constant row offset: lenslet (Iy, Ix) lives at row
//   g = m_base + Iy*Lp + Ix,  Lp = Lx + h,  m_base = h + h*Lp,
// columns Ix in [Lx, Lp) and the h rows above / below the grid stay zero, so a
// shift by D = (Dy, Dx) is the row offset Dy*Lp + Dx and every out-of-grid
// neighbour reads a zero. Output position m (0 <= m < M_out = Ly*Lp) maps to
// (Iy, Ix) = (m / Lp, m % Lp); positions with Ix >= Lx are padding.
struct Geo {
    int N, Nz, P, H, W;     // Nnum, depths, PSF width, sensor size
    int Ly, Lx, k, h, T;    // lenslet grid, PSF width in lenslets, halo, taps/axis
    int S, Spad;            // phases per lenslet N*N, padded to a multiple of 16
    int C, Cpad;            // channels Nz*S, padded to a multiple of 64
    int Lp;                 // padded row length of the lenslet grid
    int64_t m_base;         // row of lenslet (0,0) in a padded buffer
    int64_t M_out;          // output positions Ly*Lp
    int64_t M_pad;          // M_out rounded up to a multiple of 256
    int64_t rows;           // rows allocated for padded buffers
    __host__ __device__ int64_t taps() const { return (int64_t)T * T; }
};

bool make_geo(int P, int N, int Nz, int H, int W, Geo* g, std::string* why);

// FFT variant: voxels with H^T 1 below this fraction of the frame's largest are
// backprojected by direct summation; the transforms' absolute error floor
// (about 1e-7 of a tile's largest value) would dominate their update
constexpr float kLowSensitivity = 1e-3f;

// orthonormal DCT-II basis rows C_k(x; Z), k < n, x < Z (Eqs. 2-4), FP64, [n][Z]
std::vector<double> dct_table(int n, int Z);
// the same values split as FP32 pairs (hi = fl(c), lo = fl(c - hi)), for the
// row transform's double-float accumulation on the FP32 units
std::vector<float2> split_table(const std::vector<double>& t);

// ------------------------------------------------------------ device buffers --
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

// CUDA events bracketing the stages of every RL iteration while profiling is
// on; read back (and averaged) at the end of lfd_rl_iterate.
constexpr int kStageSlots = 11;  // averaged stage times (lfd_stage_times)
struct StageTimes {
    std::vector<cudaEvent_t> ev;  // 10 per iteration
    bool on = false;
    double sum_ms[kStageSlots] = {};
    int64_t count = 0;
};

struct ExactPlan;  // exact.h
struct LoPlanes;   // tc_cgemm.h
struct WidePlanes; // tc_cgemm.h

}  // namespace lfd

struct lfd_ctx {
    lfd::Geo g;
    lfd_options opt;
    int XS = 0, YS = 0;
    int device = 0;
    int sm_count = 0;
    std::string err;

    // packed PSF: [T*T][Spad][Cpad]
    float* W32 = nullptr;
    __nv_bfloat16* Wb[2] = {nullptr, nullptr};   // hi, lo
    // padded channels-last volume [rows][Cpad] (double-buffered iterate)
    float* Vp32[2] = {nullptr, nullptr};
    __nv_bfloat16* Vpb[2] = {nullptr, nullptr};  // hi, lo of the forward input
    // padded polyphase image [rows][Spad]
    float* Rp32 = nullptr;
    __nv_bfloat16* Rpb[2] = {nullptr, nullptr};
    // TF32 (direct variant): operand copies rounded to TF32 - the iterate
    // [rows][Cpad], the ratio [rows][Spad] and the transposed packed PSF
    // [T*T][Cpad][Spad] (W32 itself is rounded in place once H^T 1 is known)
    float* Vpt = nullptr;
    float* Rpt = nullptr;
    float* WT = nullptr;
    // projection outputs indexed by output position m
    float* Fwd = nullptr;        // [fwd_splits][M_pad][Spad]
    float* Bwd = nullptr;        // [bwd_splits][M_pad][Cpad]
    int fwd_splits = 1, bwd_splits = 1;
    float* invHt1 = nullptr;     // [M_pad][Cpad]
    float* ypoly = nullptr;      // [M_pad][Spad]
    // metric
    float* mip = nullptr;        // [H][W]
    float2* cosW = nullptr;      // [XS][W] FP64 basis split as FP32 hi + lo
    double* cosH = nullptr;      // [YS][H]
    double* G = nullptr;         // [H][XS]
    double* rowE2 = nullptr;     // [H] sum of mip^2 per row
    double* coef = nullptr;      // [YS][XS]
    double* flux_part = nullptr; // [Ly*Lx]
    double* hist = nullptr;      // [2][mf]: entropy, flux of the latest iteration
    double* host_pinned = nullptr;  // [4]
    double* host_hist = nullptr;    // pinned [2][mf][host_hist_n] histories
    double* host_pinned_slots = nullptr;  // pinned [2][mf] latest values per slot
    int host_hist_n = 0;
    int mf = 1;                  // frames per batch (max_frames)
    // CUDA graphs of one RL iteration (reading iterate buffer 0 or 1)
    cudaStream_t wstream = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int graph_nf = 0;
    uint64_t graph_launches = 0;  // kernels per graph replay
    // staging for host pointers
    float* stage_vol = nullptr;  // [Nz][H][W]
    float* stage_img = nullptr;  // [H][W]
    int64_t device_bytes = 0;
    lfd::StageTimes prof;
    // tensor-core path state (tcgen05), created on first use
    void* tc = nullptr;
    // FFT variant: cached PSF spectra and channel-major buffers
    void* fft = nullptr;         // FftPlan (host)
    float2* Wf = nullptr;        // [bins][S][Cf]
    float2* Xh = nullptr;        // [bins][tiles][Cf]
    float2* Yh = nullptr;        // [bins][tiles][Sf]
    __nv_bfloat16* Wp[4] = {};   // split-BF16 planes of the spectra (tensor-core contraction)
    __nv_bfloat16* Xp[4] = {};
    __nv_bfloat16* Yp[4] = {};
    void* cg = nullptr;          // tensor-core contraction state
    float* Vcm[2] = {nullptr, nullptr};  // [C][Ly][Lx]
    float* Rcm = nullptr;        // [S][Ly][Lx]
    float* Xcm = nullptr;        // [C][Ly][Lx]
    float* invcm = nullptr;      // [C][Ly][Lx]
    float* ycm = nullptr;        // [S][Ly][Lx]
    int nflux = 0;               // flux partials written per update
    float* psf_dev = nullptr;    // original PSF [Nz][N][N][P][P] (FFT variant)
    float* rimg = nullptr;       // ratio image [H][W] (FFT variant)
    lfd::ExactPlan* exact = nullptr;  // voxels backprojected exactly (FFT variant)
    lfd::LoPlanes* lo = nullptr;      // adaptive lo planes of the PSF spectra (split BF16)
    lfd::WidePlanes* wide = nullptr;  // the forward's wide-unit copy of the adaptive spectra
    int64_t spectra_bytes = 0;        // PSF spectra planes the contractions stream
    int64_t n_low = 0;
    // depth split (lfd_split_*): iterate buffer holding the current iterate
    // (-1: none loaded) and whether the other buffer holds the previous one
    int split_cur = -1;
    int split_prev = 0;
};

namespace lfd {

extern std::atomic<uint64_t> g_launches;
// compensated (Kahan) FP32 accumulation: s + c carries the sum of the added
// terms with about twice FP32's precision (the flux partial of one thread)
__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// First-fit offset allocator with coalescing (the serving arena's bookkeeping)
int64_t align256(int64_t b);
class FreeList {
  public:
    int64_t used = 0, peak = 0;
    void reset(int64_t cap) {
        free_.clear();
        taken_.clear();
        used = peak = 0;
        if (cap > 0) free_[0] = cap;
    }
    int64_t alloc(int64_t bytes);  // offset (256-byte aligned size), or -1
    bool release(int64_t off);     // false for an offset not handed out
    size_t free_blocks() const { return free_.size(); }

  private:
    std::map<int64_t, int64_t> free_;   // offset -> bytes
    std::map<int64_t, int64_t> taken_;  // offset -> bytes
};

// host-side fault injection (lfd_debug_fail_allocs): the next n device
// allocations of the library report failure without calling cudaMalloc
extern std::atomic<int> g_fail_allocs;
inline bool injected_alloc_failure() {
    int n = g_fail_allocs.load();
    while (n > 0)
        if (g_fail_allocs.compare_exchange_weak(n, n - 1)) return true;
    return false;
}

inline void count_launch(uint64_t n = 1) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// --------------------------------------------------------- kernel launchers --
// All launchers enqueue on `st` and return the launch error (cudaGetLastError).
cudaError_t launch_fill(float* p, int64_t n, float val, cudaStream_t st);
cudaError_t launch_mip_stack(const float* v, int Nz, int64_t HW, float* mip, cudaStream_t st);
cudaError_t launch_repack_psf(const float* psf, const Geo& g, float* W32,
                              __nv_bfloat16* whi, __nv_bfloat16* wlo, cudaStream_t st);
cudaError_t launch_poly_volume(const float* v, const Geo& g, float* vp32,
                               __nv_bfloat16* hi, __nv_bfloat16* lo, cudaStream_t st);
cudaError_t launch_depoly_volume(const float* vp32, int64_t row0, const Geo& g,
                                 float* v, cudaStream_t st);
cudaError_t launch_sum_depoly_volume(const float* parts, int nsplit, const Geo& g,
                                     float* v, cudaStream_t st);
cudaError_t launch_poly_image(const float* y, const Geo& g, float* dst, int64_t row0,
                              __nv_bfloat16* hi, __nv_bfloat16* lo, cudaStream_t st);
cudaError_t launch_fwd_finish_image(const float* parts, int nsplit, const Geo& g,
                                    float* y_out, cudaStream_t st);
cudaError_t launch_fwd_finish_ratio(const float* parts, int nsplit, const float* ypoly,
                                    float eps, const Geo& g, float* rp32,
                                    __nv_bfloat16* hi, __nv_bfloat16* lo, cudaStream_t st);
cudaError_t launch_inv_ht1(const float* parts, int nsplit, const Geo& g, float* inv,
                           cudaStream_t st);
cudaError_t launch_update(const float* vin, float* vout, __nv_bfloat16* hi, __nv_bfloat16* lo,
                          const float* parts, int nsplit, const float* inv, const Geo& g,
                          float* mip, double* flux_part, cudaStream_t st);
cudaError_t launch_mip(const float* vp32, const Geo& g, float* mip, cudaStream_t st);
// r[e] = y[e] / (hv[e] + eps) (0 where hv + eps <= 0), e < n
cudaError_t launch_ratio_image(const float* y, const float* hv, float eps, int64_t n, float* r,
                               cudaStream_t st);
// out[0] = sum of p[0..n) (device, fixed order)
cudaError_t launch_sum_doubles(const double* p, int64_t n, double* out, cudaStream_t st);
// DCT entropy of nf frames' MIPs (frame-major arrays: mip H*W, G H*XS, rowE2 H,
// coef XS*YS, flux_part nflux per frame); frame f writes out_entropy[f*out_stride]
// and out_flux[f*out_stride]
// launch_metric keeps kMetricScratch doubles per frame after the frames'
// coefficients: coef must hold nf * (XS * YS + kMetricScratch) doubles
constexpr int kMetricScratch = 64;
cudaError_t launch_metric(const float* mip, const float2* cosW, const double* cosH,
                          int H, int W, int XS, int YS, int l2_over_region,
                          double* G, double* rowE2, double* coef,
                          const double* flux_part, int nflux, double* out_entropy,
                          double* out_flux, cudaStream_t st, int nf = 1, int out_stride = 1);

// FP32 SIMT implicit-GEMM projections (CUDA cores)
int simt_fwd_splits(const Geo& g, int sm_count);
int simt_bwd_splits(const Geo& g, int sm_count);
cudaError_t launch_simt_forward(const float* vp32, const float* W32, const Geo& g,
                                int nsplit, float* out, cudaStream_t st);
cudaError_t launch_simt_backward(const float* rp32, const float* W32, const Geo& g,
                                 int nsplit, float* out, cudaStream_t st);

}  // namespace lfd
