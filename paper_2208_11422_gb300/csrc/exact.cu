// Exact backprojection of the FFT variant's low-sensitivity voxels: the
// backprojection of Section 2.1 written out as window sums,
//   (H^T r)[z][ip][jp] = sum_{mi, mj} r[ip - c + mi][jp - c + mj] K[mi][mj],
// K the PSF tile of the voxel's depth and phase (ty, tx), c = (P - 1) / 2,
// the window clipped to the sensor (zero outside).
//
// At the sensor's borders these voxels come in runs: a lenslet row (Iy fixed)
// or column (Ix fixed) of one channel (z, ty, tx). A row run shares K and,
// PSF row by PSF row, one image row. A block (or a warp) owns a piece of a
// run: for each PSF row mi it stages the image-row segment the piece's
// windows touch in shared memory (zeros outside the sensor), every lane holds
// K[mi][lane + 32 s] in registers, and voxel v adds
//   sum_s rs[(jp_v - jp_first) + lane + 32 s] * K[mi][lane + 32 s],
// one shared-memory load and one FMA per product, the next image row and PSF
// row already in flight. Runs of 8 or more voxels are cut into pieces of at
// most 24 voxels on four warps; shorter runs and lone voxels are pieces of one
// warp. Pieces are sorted by cost and dealt to a grid of one wave (block b
// takes pieces b, b + grid, ...), so no SM is left with a long tail. A column
// run is a row run of the transposed problem (transposed ratio image,
// transposed PSF tile). PSF rows wider than 512 taps take the
// one-warp-per-voxel kernel (k_exact_bwd).
#include <algorithm>
#include <cstring>
#include <random>
#include <new>
#include <unordered_map>
#include <vector>

#include "exact.h"
#include "fft_proj.h"

namespace lfd {

namespace {

// long runs (>= kMinLong voxels): pieces of at most kLongWarps * kLongVpw
// voxels on kLongWarps warps; short runs and single voxels: one warp each
constexpr int kLongWarps = 4, kLongVpw = 6, kMaxPiece = kLongWarps * kLongVpw;  // 24 voxels
constexpr int kMinLong = 8;
constexpr int kShortVpw = kMinLong - 1;
constexpr int kNsMax = 16;               // PSF rows up to 512 taps (ns = ceil(P / 32) <= 16)
constexpr int kLongFill = 8, kShortFill = 16;  // image-row floats per thread
// PSF rows per pass between barriers (long pieces): two measured 0.696 against
// 0.685 ms at the large frame (128 instead of 72 registers, 16 instead of 28
// warps per SM)
constexpr int kLongRps = 1;
constexpr int kLongSpan = 32 * kLongWarps * kLongFill, kShortSpan = 32 * kShortFill;

struct ExactRun {
    int64_t ktile;  // float offset of the run's PSF tile (psf, or psfT for a column run)
    int orient;     // 0: along a lenslet row (positions Ix), 1: along a column (positions Iy)
    int fixed;      // Iy (row run) or Ix (column run)
    int pf, pp;     // phase along the fixed axis and along the run: (ty, tx) or (tx, ty)
    int first, count;
};

template <int WARPS>
__device__ __forceinline__ void piece_sync() {
    if constexpr (WARPS == 1) __syncwarp();
    else __syncthreads();
}

// One piece of a run with WARPS warps, VPW voxel slots per warp, NS =
// ceil(P / 32) chunks of a PSF row per lane, and image-row segments of up to
// 32 WARPS FILL floats, RPS PSF rows (and image rows) per pass between two
// block barriers. The next pass's PSF rows and image rows are loaded into
// registers while the current ones are summed.
template <int NS, int WARPS, int VPW, int FILL, int RPS>
__device__ void exact_piece(const ExactRun& R, int f, const int* __restrict__ pos,
                            const int64_t* __restrict__ out, const float* __restrict__ rimg,
                            const float* __restrict__ rimgT, const float* __restrict__ psf,
                            const float* __restrict__ psfT, const Geo& g, float* __restrict__ xcm,
                            float* rs) {
    constexpr int T = 32 * WARPS;
    const bool tr = R.orient != 0;
    const int Hh = tr ? g.W : g.H, Ww = tr ? g.H : g.W;
    const float* img = (tr ? rimgT : rimg) + (int64_t)f * g.H * g.W;
    const float* K = (tr ? psfT : psf) + R.ktile;
    const int P = g.P, c0 = (P - 1) / 2;
    const int ip = R.fixed * g.N + R.pf;
    const int mi0 = max(0, c0 - ip), mi1 = min(P, Hh + c0 - ip);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j0 = pos[R.first] * g.N + R.pp - c0;
    const int span = (pos[R.first + R.count - 1] - pos[R.first]) * g.N + 32 * NS;
    int off[VPW];
#pragma unroll
    for (int k = 0; k < VPW; ++k) {
        const int v = warp + WARPS * k;
        off[k] = v < R.count ? (pos[R.first + v] - pos[R.first]) * g.N : 0;
    }
    float acc[VPW];
#pragma unroll
    for (int k = 0; k < VPW; ++k) acc[k] = 0.f;

    float nxt[RPS][FILL], knx[RPS][NS];
    auto fetch = [&](int m) {  // image rows and PSF rows m .. m + RPS - 1 into registers
#pragma unroll
        for (int r = 0; r < RPS; ++r) {
            const int mi = m + r;
            const bool in = mi < mi1;
            const float* row = img + (int64_t)(ip - c0 + (in ? mi : m)) * Ww;
#pragma unroll
            for (int u = 0; u < FILL; ++u) {
                const int e = threadIdx.x + u * T, col = j0 + e;
                nxt[r][u] = (in && e < span && col >= 0 && col < Ww) ? row[col] : 0.f;
            }
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                const int mj = lane + 32 * s;
                knx[r][s] = (in && mj < P) ? K[(int64_t)mi * P + mj] : 0.f;
            }
        }
    };
    if (mi0 < mi1) fetch(mi0);
    for (int mi = mi0; mi < mi1; mi += RPS) {
        piece_sync<WARPS>();  // the previous pass's products are done
#pragma unroll
        for (int r = 0; r < RPS; ++r)
#pragma unroll
            for (int u = 0; u < FILL; ++u) {
                const int e = threadIdx.x + u * T;
                if (e < span) rs[r * span + e] = nxt[r][u];
            }
        float kr[RPS][NS];
#pragma unroll
        for (int r = 0; r < RPS; ++r)
#pragma unroll
            for (int s = 0; s < NS; ++s) kr[r][s] = knx[r][s];
        piece_sync<WARPS>();
        if (mi + RPS < mi1) fetch(mi + RPS);
#pragma unroll
        for (int r = 0; r < RPS; ++r) {
            if (mi + r >= mi1) break;
#pragma unroll
            for (int k = 0; k < VPW; ++k) {
                if (warp + WARPS * k < R.count) {
                    const float* q = rs + r * span + off[k] + lane;
#pragma unroll
                    for (int s = 0; s < NS; ++s) acc[k] = fmaf(q[32 * s], kr[r][s], acc[k]);
                }
            }
        }
    }
    float* x = xcm + (int64_t)f * g.C * g.Ly * g.Lx;
#pragma unroll
    for (int k = 0; k < VPW; ++k) {
        const int v = warp + WARPS * k;
        float a = acc[k];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (v < R.count && lane == 0) x[out[R.first + v]] = a;
    }
}

// pieces sorted by cost; block b of the grid takes pieces b, b + gridDim.x, ...
template <int NS, int WARPS, int VPW, int FILL, int RPS>
__global__ void __launch_bounds__(32 * WARPS) k_exact_runs(const ExactRun* __restrict__ runs, int nruns,
                                                           const int* __restrict__ pos,
                                                           const int64_t* __restrict__ out,
                                                           const float* __restrict__ rimg,
                                                           const float* __restrict__ rimgT,
                                                           const float* __restrict__ psf,
                                                           const float* __restrict__ psfT, Geo g,
                                                           float* __restrict__ xcm) {
    extern __shared__ float rs[];
    for (int b = blockIdx.x; b < nruns; b += gridDim.x) {
        const ExactRun R = runs[b];
        exact_piece<NS, WARPS, VPW, FILL, RPS>(R, blockIdx.y, pos, out, rimg, rimgT, psf, psfT, g, xcm, rs);
        piece_sync<WARPS>();  // rs is reused by the next piece
    }
}

using RunsKernel = void (*)(const ExactRun*, int, const int*, const int64_t*, const float*, const float*,
                            const float*, const float*, Geo, float*);

template <int NS, int WARPS, int VPW, int FILL, int RPS>
RunsKernel runs_kernel_n(int ns) {
    if constexpr (NS > kNsMax) {
        return nullptr;
    } else {
        return ns == NS ? k_exact_runs<NS, WARPS, VPW, FILL, RPS> : runs_kernel_n<NS + 1, WARPS, VPW, FILL, RPS>(ns);
    }
}

// dst[f][x][y] = src[f][y][x] for [nf][H][W] images, 32 x 32 tiles
__global__ void k_transpose_images(const float* __restrict__ src, int H, int W, float* __restrict__ dst) {
    __shared__ float t[32][33];
    const int64_t fo = (int64_t)blockIdx.z * H * W;
    const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int y = y0 + i, x = x0 + threadIdx.x;
        if (y < H && x < W) t[i][threadIdx.x] = src[fo + (int64_t)y * W + x];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int x = x0 + i, y = y0 + threadIdx.x;
        if (x < W && y < H) dst[fo + (int64_t)x * H + y] = t[threadIdx.x][i];
    }
}

// psfT[j] = transpose of the P x P PSF tile of channel chan[j]
__global__ void k_transpose_tiles(const float* __restrict__ psf, const int* __restrict__ chan, int P,
                                  float* __restrict__ psfT) {
    __shared__ float t[32][33];
    const float* src = psf + (int64_t)chan[blockIdx.z] * P * P;
    float* dst = psfT + (int64_t)blockIdx.z * P * P;
    const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int y = y0 + i, x = x0 + threadIdx.x;
        if (y < P && x < P) t[i][threadIdx.x] = src[(int64_t)y * P + x];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int x = x0 + i, y = y0 + threadIdx.x;
        if (x < P && y < P) dst[(int64_t)x * P + y] = t[threadIdx.x][i];
    }
}

cudaError_t plan_alloc(void** p, size_t bytes, int64_t* total) {
    if (injected_alloc_failure()) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) *total += (int64_t)bytes;
    return e;
}

}  // namespace

struct ExactPlan {
    Geo g{};
    int max_frames = 0;
    const float* psf = nullptr;
    ExactRun* runs = nullptr;   // the long pieces, then the short ones
    int nlong = 0, nshort = 0;
    int* pos = nullptr;
    int64_t* out = nullptr;
    int64_t in_runs = 0;
    int64_t* single = nullptr;  // voxels summed one warp each (PSF rows over 512 taps)
    int64_t nsingle = 0;
    float* psfT = nullptr;
    float* rimgT = nullptr;
    int span_long = 0, span_short = 0;  // largest staged image row of a piece
    RunsKernel kern_long = nullptr, kern_short = nullptr;
    int slots_long = 0, slots_short = 0;  // resident blocks on the device
};

namespace {
cudaError_t slots_for(RunsKernel k, int threads, size_t smem, int* slots) {
    int per_sm = 0, dev = 0, sms = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
        (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem)) != cudaSuccess)
        return e;
    *slots = std::max(1, per_sm * sms);
    return cudaSuccess;
}
}  // namespace

namespace {

// The host half of a plan: the pieces (long ones first, each kind sorted by
// cost), their voxels' positions along the run and output indices, the voxels
// left to one warp each, and the channels whose PSF tile is transposed.
struct RunPlan {
    std::vector<ExactRun> runs;
    int nlong = 0, nshort = 0;
    std::vector<int> pos;
    std::vector<int64_t> out;
    std::vector<int64_t> single;
    std::vector<int> tchan;
    int span_long = 0, span_short = 0;
};

RunPlan build_runs(const int64_t* low, int64_t n, const Geo& g) {
    RunPlan rp;
    const int64_t L2 = (int64_t)g.Ly * g.Lx;
    const int ns = (g.P + 31) / 32;
    // run lengths along rows (c, Iy) and columns (c, Ix); each voxel joins the
    // longer of its two runs
    std::unordered_map<int64_t, int> nrow, ncol;
    std::vector<int> cs(n), iys(n), ixs(n);
    for (int64_t i = 0; i < n; ++i) {
        const int64_t idx = low[i];
        cs[i] = (int)(idx / L2);
        iys[i] = (int)((idx % L2) / g.Lx);
        ixs[i] = (int)(idx % g.Lx);
        ++nrow[(int64_t)cs[i] * g.Ly + iys[i]];
        ++ncol[(int64_t)cs[i] * g.Lx + ixs[i]];
    }
    struct Item {
        int orient, c, fixed, pos;
        int64_t idx;
    };
    std::vector<Item> items;
    items.reserve(n);
    const bool runs_ok = ns <= kNsMax;  // else every voxel takes the one-warp-per-voxel kernel
    for (int64_t i = 0; i < n; ++i) {
        const int lr = nrow[(int64_t)cs[i] * g.Ly + iys[i]], lc = ncol[(int64_t)cs[i] * g.Lx + ixs[i]];
        if (!runs_ok) {
            rp.single.push_back(low[i]);
            continue;
        }
        if (lr >= lc) items.push_back({0, cs[i], iys[i], ixs[i], low[i]});
        else items.push_back({1, cs[i], ixs[i], iys[i], low[i]});
    }
    std::sort(items.begin(), items.end(), [](const Item& a, const Item& b) {
        if (a.orient != b.orient) return a.orient < b.orient;
        if (a.c != b.c) return a.c < b.c;
        if (a.fixed != b.fixed) return a.fixed < b.fixed;
        return a.pos < b.pos;
    });
    std::vector<ExactRun> shorts;
    std::unordered_map<int, int> tslot;
    for (size_t a = 0; a < items.size();) {
        size_t b = a;
        while (b < items.size() && items[b].orient == items[a].orient && items[b].c == items[a].c &&
               items[b].fixed == items[a].fixed)
            ++b;
        const bool is_long = b - a >= (size_t)kMinLong;
        const Item& h = items[a];
        const int t = h.c % g.S, ty = t / g.N, tx = t % g.N;
        int64_t ktile = (int64_t)h.c * g.P * g.P;
        if (h.orient) {
            auto it = tslot.find(h.c);
            if (it == tslot.end()) {
                it = tslot.emplace(h.c, (int)rp.tchan.size()).first;
                rp.tchan.push_back(h.c);
            }
            ktile = (int64_t)it->second * g.P * g.P;
        }
        // pieces of at most kMaxPiece (long) or kShortVpw (short) voxels
        // whose staged row segment fits
        const size_t cap = is_long ? kMaxPiece : kShortVpw;
        const int span_cap = is_long ? kLongSpan : kShortSpan;
        for (size_t s = a; s < b;) {
            size_t e = s + 1;
            while (e < b && e + 1 - s <= cap && (items[e].pos - items[s].pos) * g.N + 32 * ns <= span_cap)
                ++e;
            ExactRun r{};
            r.ktile = ktile;
            r.orient = h.orient;
            r.fixed = h.fixed;
            r.pf = h.orient ? tx : ty;
            r.pp = h.orient ? ty : tx;
            r.first = (int)rp.pos.size();
            r.count = (int)(e - s);
            for (size_t i = s; i < e; ++i) {
                rp.pos.push_back(items[i].pos);
                rp.out.push_back(items[i].idx);
            }
            const int span = (items[e - 1].pos - items[s].pos) * g.N + 32 * ns;
            int& sm = is_long ? rp.span_long : rp.span_short;
            sm = std::max(sm, span);
            (is_long ? rp.runs : shorts).push_back(r);
            s = e;
        }
        a = b;
    }
    std::sort(rp.single.begin(), rp.single.end());
    // costliest pieces first (voxels x PSF rows inside the sensor), so that the
    // grid's block-stride deal ends evenly
    auto cost = [&](const ExactRun& r) {
        const int ip = r.fixed * g.N + r.pf, c0 = (g.P - 1) / 2, Hh = r.orient ? g.W : g.H;
        return (int64_t)r.count * std::max(0, std::min(g.P, Hh + c0 - ip) - std::max(0, c0 - ip));
    };
    auto by_cost = [&](const ExactRun& a, const ExactRun& b) { return cost(a) > cost(b); };
    std::stable_sort(rp.runs.begin(), rp.runs.end(), by_cost);
    std::stable_sort(shorts.begin(), shorts.end(), by_cost);
    rp.nlong = (int)rp.runs.size();
    rp.nshort = (int)shorts.size();
    rp.runs.insert(rp.runs.end(), shorts.begin(), shorts.end());
    return rp;
}

}  // namespace

cudaError_t exact_plan_create(const int64_t* low, int64_t n, const Geo& g, const float* psf, int max_frames,
                              cudaStream_t st, ExactPlan** out, int64_t* bytes, std::string* why) {
    *out = nullptr;
    ExactPlan* p = new (std::nothrow) ExactPlan();
    if (!p) return cudaErrorMemoryAllocation;
    p->g = g;
    p->max_frames = max_frames;
    p->psf = psf;
    const int ns = (g.P + 31) / 32;
    RunPlan rp = build_runs(low, n, g);
    const std::vector<ExactRun>& runs = rp.runs;
    const std::vector<int>& pos = rp.pos;
    const std::vector<int64_t>& outs = rp.out;
    const std::vector<int64_t>& single = rp.single;
    const std::vector<int>& tchan = rp.tchan;
    p->nlong = rp.nlong;
    p->nshort = rp.nshort;
    p->span_long = rp.span_long;
    p->span_short = rp.span_short;
    p->in_runs = (int64_t)pos.size();
    p->nsingle = (int64_t)single.size();
    int64_t total = 0;
    cudaError_t e = cudaSuccess;
    auto fail = [&](const char* what) {
        if (why) *why = std::string("exact correction plan: ") + what + ": " + cudaGetErrorString(e);
        *bytes += total;
        *out = p;  // the caller destroys it
        return e;
    };
    if (!runs.empty()) {
        if ((e = plan_alloc((void**)&p->runs, sizeof(ExactRun) * runs.size(), &total)) != cudaSuccess ||
            (e = plan_alloc((void**)&p->pos, sizeof(int) * pos.size(), &total)) != cudaSuccess ||
            (e = plan_alloc((void**)&p->out, sizeof(int64_t) * outs.size(), &total)) != cudaSuccess)
            return fail("allocation");
        if ((e = cudaMemcpyAsync(p->runs, runs.data(), sizeof(ExactRun) * runs.size(), cudaMemcpyHostToDevice,
                                 st)) != cudaSuccess ||
            (e = cudaMemcpyAsync(p->pos, pos.data(), sizeof(int) * pos.size(), cudaMemcpyHostToDevice, st)) !=
                cudaSuccess ||
            (e = cudaMemcpyAsync(p->out, outs.data(), sizeof(int64_t) * outs.size(), cudaMemcpyHostToDevice,
                                 st)) != cudaSuccess)
            return fail("upload");
        p->kern_long = runs_kernel_n<1, kLongWarps, kLongVpw, kLongFill, kLongRps>(ns);
        p->kern_short = runs_kernel_n<1, 1, kShortVpw, kShortFill, 1>(ns);
        if ((p->nlong && (e = slots_for(p->kern_long, 32 * kLongWarps, sizeof(float) * kLongRps * p->span_long,
                                        &p->slots_long)) != cudaSuccess) ||
            (p->nshort && (e = slots_for(p->kern_short, 32, sizeof(float) * p->span_short,
                                         &p->slots_short)) != cudaSuccess))
            return fail("occupancy query");
    }
    if (!tchan.empty()) {
        int* dchan = nullptr;
        if ((e = plan_alloc((void**)&p->psfT, sizeof(float) * tchan.size() * g.P * g.P, &total)) != cudaSuccess ||
            (e = plan_alloc((void**)&p->rimgT, sizeof(float) * max_frames * (size_t)g.H * g.W, &total)) !=
                cudaSuccess)
            return fail("allocation");
        if ((e = cudaMalloc((void**)&dchan, sizeof(int) * tchan.size())) != cudaSuccess) return fail("allocation");
        e = cudaMemcpyAsync(dchan, tchan.data(), sizeof(int) * tchan.size(), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) {
            const dim3 grid((g.P + 31) / 32, (g.P + 31) / 32, (unsigned)tchan.size());
            k_transpose_tiles<<<grid, dim3(32, 8), 0, st>>>(psf, dchan, g.P, p->psfT);
            count_launch();
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        cudaFree(dchan);
        if (e != cudaSuccess) return fail("PSF tile transpose");
    }
    if (p->nsingle) {
        if ((e = plan_alloc((void**)&p->single, sizeof(int64_t) * single.size(), &total)) != cudaSuccess)
            return fail("allocation");
        if ((e = cudaMemcpyAsync(p->single, single.data(), sizeof(int64_t) * single.size(),
                                 cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return fail("upload");
    }
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return fail("upload");
    *bytes += total;
    *out = p;
    return cudaSuccess;
}

cudaError_t exact_bwd(ExactPlan* p, int nf, const float* rimg, float* xcm, cudaStream_t st) {
    if (!p || nf <= 0) return cudaSuccess;
    if (nf > p->max_frames) return cudaErrorInvalidValue;
    const Geo& g = p->g;
    if (p->rimgT) {
        const dim3 grid((g.W + 31) / 32, (g.H + 31) / 32, (unsigned)nf);
        k_transpose_images<<<grid, dim3(32, 8), 0, st>>>(rimg, g.H, g.W, p->rimgT);
        count_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (p->nlong) {
        const int gx = std::min(p->nlong, std::max(1, p->slots_long / nf));
        p->kern_long<<<dim3((unsigned)gx, (unsigned)nf), 32 * kLongWarps, sizeof(float) * kLongRps * p->span_long,
                       st>>>(
            p->runs, p->nlong, p->pos, p->out, rimg, p->rimgT, p->psf, p->psfT, g, xcm);
        count_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (p->nshort) {
        const int gx = std::min(p->nshort, std::max(1, p->slots_short / nf));
        p->kern_short<<<dim3((unsigned)gx, (unsigned)nf), 32, sizeof(float) * p->span_short, st>>>(
            p->runs + p->nlong, p->nshort, p->pos, p->out, rimg, p->rimgT, p->psf, p->psfT, g, xcm);
        count_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return launch_exact_bwd(p->single, p->nsingle, nf, rimg, p->psf, g, xcm, st);
}

void exact_plan_counts(const ExactPlan* p, int64_t* in_runs, int64_t* runs, int64_t* single) {
    if (in_runs) *in_runs = p ? p->in_runs : 0;
    if (runs) *runs = p ? p->nlong + p->nshort : 0;
    if (single) *single = p ? p->nsingle : 0;
}

void exact_plan_destroy(ExactPlan* p) {
    if (!p) return;
    void* ptrs[] = {p->runs, p->pos, p->out, p->single, p->psfT, p->rimgT};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    delete p;
}

}  // namespace lfd

// Host-only check of the run plan on a seeded synthetic list (border bands,
// corner blocks, scattered voxels): every voxel is summed exactly once, a
// piece holds voxels of one channel along one lenslet row or column in
// increasing order, within the piece and staging limits, its PSF tile offset
// names the voxel's channel (or its transposed copy), and the long pieces
// come first, each kind sorted by cost.
extern "C" lfd_status lfd_selftest_exact_runs(int seed, int N, int Nz, int k, int L) {
    using namespace lfd;
    if (N < 1 || N % 2 == 0 || Nz < 1 || k < 1 || k % 2 == 0 || L < 1 || L > 256) return LFD_EINVAL;
    Geo g{};
    std::string why;
    if (!make_geo(k * N, N, Nz, L * N, L * N, &g, &why)) return LFD_EINVAL;
    std::mt19937_64 rng((uint64_t)seed);
    const int64_t L2 = (int64_t)g.Ly * g.Lx;
    std::vector<char> mark((size_t)g.C * L2, 0);
    for (int c = 0; c < g.C; ++c) {
        const int kind = (int)(rng() % 5);
        const int w = 1 + (int)(rng() % 3);
        for (int iy = 0; iy < g.Ly; ++iy)
            for (int ix = 0; ix < g.Lx; ++ix) {
                bool on = false;
                if (kind == 0) on = iy < w;                             // top band
                if (kind == 1) on = ix >= g.Lx - w;                     // right band
                if (kind == 2) on = iy < w + 2 && ix < w + 2;           // corner block
                if (kind == 3) on = rng() % 97 == 0;                    // scattered
                if (on) mark[(size_t)c * L2 + (size_t)iy * g.Lx + ix] = 1;
            }
    }
    std::vector<int64_t> low;
    for (size_t i = 0; i < mark.size(); ++i)
        if (mark[i]) low.push_back((int64_t)i);
    const RunPlan rp = build_runs(low.data(), (int64_t)low.size(), g);
    const int ns = (g.P + 31) / 32;
    std::vector<char> seen(mark.size(), 0);
    auto cost = [&](const ExactRun& r) {
        const int ip = r.fixed * g.N + r.pf, c0 = (g.P - 1) / 2, Hh = r.orient ? g.W : g.H;
        return (int64_t)r.count * std::max(0, std::min(g.P, Hh + c0 - ip) - std::max(0, c0 - ip));
    };
    if (rp.nlong + rp.nshort != (int)rp.runs.size()) return LFD_EINTERNAL;
    for (size_t r = 0; r < rp.runs.size(); ++r) {
        const ExactRun& R = rp.runs[r];
        const bool is_long = (int)r < rp.nlong;
        if (R.count < 1 || R.count > (is_long ? kMaxPiece : kShortVpw)) return LFD_EINTERNAL;
        if (r > 0 && (int)r != rp.nlong && cost(rp.runs[r - 1]) < cost(R)) return LFD_EINTERNAL;
        const int span = (rp.pos[R.first + R.count - 1] - rp.pos[R.first]) * g.N + 32 * ns;
        if (span > (is_long ? rp.span_long : rp.span_short) || span > (is_long ? kLongSpan : kShortSpan))
            return LFD_EINTERNAL;
        for (int v = 0; v < R.count; ++v) {
            const int64_t idx = rp.out[R.first + v];
            if (idx < 0 || idx >= (int64_t)mark.size() || !mark[idx] || seen[idx]) return LFD_EINTERNAL;
            seen[idx] = 1;
            const int c = (int)(idx / L2), iy = (int)((idx % L2) / g.Lx), ix = (int)(idx % g.Lx);
            const int t = c % g.S, ty = t / g.N, tx = t % g.N;
            const int fixed = R.orient ? ix : iy, along = R.orient ? iy : ix;
            if (R.fixed != fixed || rp.pos[R.first + v] != along) return LFD_EINTERNAL;
            if (R.pf != (R.orient ? tx : ty) || R.pp != (R.orient ? ty : tx)) return LFD_EINTERNAL;
            if (v > 0 && rp.pos[R.first + v] <= rp.pos[R.first + v - 1]) return LFD_EINTERNAL;
            const int64_t tile = R.ktile / ((int64_t)g.P * g.P);
            if (R.ktile % ((int64_t)g.P * g.P) != 0) return LFD_EINTERNAL;
            if (R.orient ? (tile >= (int64_t)rp.tchan.size() || rp.tchan[tile] != c) : tile != c)
                return LFD_EINTERNAL;
        }
    }
    for (int64_t idx : rp.single) {
        if (!mark[idx] || seen[idx]) return LFD_EINTERNAL;
        seen[idx] = 1;
    }
    for (size_t i = 0; i < mark.size(); ++i)
        if (mark[i] != seen[i]) return LFD_EINTERNAL;
    return LFD_OK;
}
