// Split-BF16 complex contractions of the FFT variant on the tcgen05 tensor
// cores (per frequency bin of the overlap-save transforms):
//
//   forward  Yh[bin][t][s] = sum_c       Wf[bin][s][c]  Xh[bin][t][c]
//   adjoint  Xh[bin][t][c] = sum_s  conj(Wf[bin][s][c]) Yh[bin][t][s]
//
// Every complex operand is held as four BF16 planes (real hi, real lo, imag
// hi, imag lo; x = hi + lo) and every complex product becomes real MMAs:
//   forward  re += Wr Xr - Wi Xi,   im += Wr Xi + Wi Xr
//   adjoint  re += Wr Yr + Wi Yi,   im += Wr Yi - Wi Yr
// each of them in three passes hi*hi + hi*lo + lo*hi (negation through the
// instruction descriptor). With BF16 PSF spectra (no lo planes of Wf) the
// passes are hi*hi + hi*lo: the PSF spectra are rounded once, the transformed
// data still carry hi + lo, and the spectra stream is 4 bytes per complex
// value instead of 8. One block owns 128 output rows (phases s for the
// forward, channels c for the adjoint) by a chunk of 16, 32 or 64 columns
// (frame x tile) of one bin, so a spectra tile is loaded once for up to 64
// columns; units are ordered bin-major so the blocks working on one bin share
// its spectra in L2. Its K loop streams 64-wide blocks of all eight planes
// through a TMA ring (3 stages for 16 columns, 2 for wider chunks). The
// accumulators (real and imaginary, one chunk of columns each) alternate
// between two TMEM buffers so the drain of one chunk overlaps the next; chains
// are cut every 64 k-blocks (1536 MMA steps) and added into the FP32 output at
// L2 (the same rounding control as the direct projections). The spectra (all
// of Wf) are read once per projection while the columns fit one chunk: the
// kernel is bound by HBM bandwidth.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <new>

#include "tc_cgemm.h"
#include "tc_ptx.h"

namespace lfd {
namespace {

using namespace tcx;

constexpr int kPlaneA = 128 * 64 * 2;  // 16 KB
constexpr int kThreads = 192;
constexpr int kChunkKb = 64;  // 64 k-blocks x 4 k-steps x 3 passes x 2 = 1536 MMA steps

// Shapes of a unit of NG groups of 16 columns (NG = 1, 2 or 4). SW: the PSF
// spectra as four planes (split BF16, three products per term); otherwise as
// their two hi planes (BF16 spectra, two products per term: W x_hi + W x_lo).
template <int NG, bool SW>
struct Cg {
    static constexpr int N = 16 * NG;                        // MMA N
    static constexpr int NA = SW ? 4 : 2;                    // PSF planes per stage
    static constexpr int NP = SW ? 3 : 2;                    // products per term
    static constexpr int kPlaneB = N * 64 * 2;               // 2, 4 or 8 KB
    static constexpr int kStageBytes = NA * kPlaneA + 4 * kPlaneB;
    static constexpr int kStages = (232448 - 1280) / kStageBytes < 6 ? (232448 - 1280) / kStageBytes : 6;
    static constexpr int kSmemBytes = kStages * kStageBytes + 1024 + 256;
    static constexpr uint32_t kTmemCols = 64 * NG;           // 2 buffers x (real, imag) x N
    static_assert(kStages >= 2 && kSmemBytes <= 232448, "stage ring exceeds the shared memory of a block");
};

struct CgArgs {
    int nbins;
    int ncol;          // output columns (frames x tiles) of this launch
    int nchunk;        // column chunks of 16 x NG
    int mtiles;        // row tiles of 128 per bin
    int nkb;           // k-blocks of 64 per unit
    int nrows;         // valid rows (S or C)
    int ld;            // row length of the output (Sf or Cf)
    float2* out;       // [bins][ntile][ld]
    int* err;
};

template <bool ADJ, int NG, bool SW>
__global__ void __launch_bounds__(kThreads, 1)
k_tc_cgemm(const __grid_constant__ CUtensorMap a0, const __grid_constant__ CUtensorMap a1,
           const __grid_constant__ CUtensorMap a2, const __grid_constant__ CUtensorMap a3,
           const __grid_constant__ CUtensorMap b0, const __grid_constant__ CUtensorMap b1,
           const __grid_constant__ CUtensorMap b2, const __grid_constant__ CUtensorMap b3,
           const CgArgs a) {
    using G = Cg<NG, SW>;
    constexpr int kStages = G::kStages, kStageBytes = G::kStageBytes;
    constexpr int kPlaneB = G::kPlaneB, N = G::N, NA = G::NA;
    constexpr uint32_t kTmemCols = G::kTmemCols;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t sbase = (raw + 1023u) & ~1023u;
    uint8_t* smem = smem_raw + (sbase - raw);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes);
    uint64_t* empty = full + kStages;
    uint64_t* acc_full = empty + kStages;   // [2]
    uint64_t* acc_empty = acc_full + 2;     // [2]
    uint64_t* mma_done = acc_empty + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_done + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    volatile int* consumed_ctr = reinterpret_cast<volatile int*>(tmem_slot + 2);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_units = a.nbins * a.nchunk * a.mtiles;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 128);
        }
        mbar_init(mma_done, 1);
        *abort_flag = 0;
        *consumed_ctr = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ------------------------------------------------- TMA producer --
            const CUtensorMap* A[4] = {&a0, &a1, &a2, &a3};
            const CUtensorMap* B[4] = {&b0, &b1, &b2, &b3};
            int stage = 0, issued = 0;
            uint32_t phase = 0;
            bool ok = true;
            for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
                const int bin = u / (a.nchunk * a.mtiles), rem = u % (a.nchunk * a.mtiles);
                const int q = rem / a.mtiles, mt = rem % a.mtiles;
                for (int kb = 0; kb < a.nkb && ok; ++kb) {
                    if (!mbar_wait(&empty[stage], phase ^ 1u, abort_flag, a.err, 11)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(&full[stage], kStageBytes);
                    const uint32_t sA = sbase + stage * kStageBytes, sB = sA + NA * kPlaneA;
#pragma unroll
                    for (int i = 0; i < NA; ++i) {
                        if (ADJ) {  // MN-major: two 64-channel atoms of 64 phases
                            tma_3d(sA + i * kPlaneA, A[i], mt * 128, kb * 64, bin, &full[stage]);
                            tma_3d(sA + i * kPlaneA + 8192, A[i], mt * 128 + 64, kb * 64, bin, &full[stage]);
                        } else {
                            tma_3d(sA + i * kPlaneA, A[i], kb * 64, mt * 128, bin, &full[stage]);
                        }
                    }
#pragma unroll
                    for (int i = 0; i < 4; ++i)  // 8 channels x 1 bin x N columns x 8 groups: [group][column][8]
                        tma_4d(sB + i * kPlaneB, B[i], 0, bin, q * N, kb * 8, &full[stage]);
                    ++issued;
                    if (++stage == kStages) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (!ok)
                for (int i = *consumed_ctr; i < issued; ++i)
                    mbar_wait_drain(&full[i % kStages], (uint32_t)((i / kStages) & 1));
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------------------------------------------- MMA issuer --
            const uint32_t id_p = idesc_bf16(128, N, false, ADJ, false);
            const uint32_t id_n = idesc_bf16(128, N, false, ADJ, true);
            int stage = 0, consumed = 0, ci = 0;
            uint32_t phase = 0;
            bool ok = true;
            for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
                for (int c0 = 0; c0 < a.nkb && ok; c0 += kChunkKb, ++ci) {
                    const int c1 = min(a.nkb, c0 + kChunkKb);
                    const int buf = ci & 1;
                    if (ci >= 2 &&
                        !mbar_wait(&acc_empty[buf], (uint32_t)(((ci - 2) >> 1) & 1), abort_flag, a.err, 12)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t dR = tmem + buf * 2 * N, dI = dR + N;
                    bool first = true;
                    for (int kb = c0; kb < c1 && ok; ++kb) {
                        if (!mbar_wait(&full[stage], phase, abort_flag, a.err, 13)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t sA = sbase + stage * kStageBytes, sB = sA + NA * kPlaneA;
#pragma unroll
                        for (int ks = 0; ks < 4; ++ks) {
                            // B planes: 0 real hi, 1 real lo, 2 imag hi, 3 imag lo; A planes
                            // the same (SW), or 0 real hi, 1 imag hi
                            uint64_t ad[NA], bd[4];
#pragma unroll
                            for (int i = 0; i < NA; ++i)
                                ad[i] = ADJ ? sdesc(sA + i * kPlaneA + ks * 2048, 8192, 1024)
                                            : sdesc(sA + i * kPlaneA + ks * 32, 16, 1024);
#pragma unroll
                            for (int i = 0; i < 4; ++i)  // K = 16 per MMA: groups 2ks, 2ks+1 (N x 16 B
                                                         // apart); 8-column core matrices 128 B apart
                                bd[i] = sdesc_noswz(sB + i * kPlaneB + ks * 2 * N * 16, N * 16, 128);
#pragma unroll
                            for (int p = 0; p < G::NP; ++p) {
                                // SW: (hi, hi), (hi, lo), (lo, hi); else (hi, hi), (hi, lo)
                                const int ia = (SW && p == 2) ? 1 : 0;
                                const int ib = p == 1 ? 1 : 0;
                                const uint64_t wr = ad[ia], wi = ad[SW ? 2 + ia : 1];
                                const uint32_t acc0 = (first && ks == 0 && p == 0) ? 0u : 1u;
                                if (!ADJ) {
                                    umma_bf16(dR, wr, bd[ib], id_p, acc0);          // + Wr Xr
                                    umma_bf16(dR, wi, bd[2 + ib], id_n, 1u);        // - Wi Xi
                                    umma_bf16(dI, wr, bd[2 + ib], id_p, acc0);      // + Wr Xi
                                    umma_bf16(dI, wi, bd[ib], id_p, 1u);            // + Wi Xr
                                } else {
                                    umma_bf16(dR, wr, bd[ib], id_p, acc0);          // + Wr Yr
                                    umma_bf16(dR, wi, bd[2 + ib], id_p, 1u);        // + Wi Yi
                                    umma_bf16(dI, wr, bd[2 + ib], id_p, acc0);      // + Wr Yi
                                    umma_bf16(dI, wi, bd[ib], id_n, 1u);            // - Wi Yr
                                }
                            }
                        }
                        first = false;
                        umma_commit(&empty[stage]);
                        *consumed_ctr = ++consumed;
                        if (++stage == kStages) {
                            stage = 0;
                            phase ^= 1u;
                        }
                    }
                    if (ok) umma_commit(&acc_full[buf]);
                }
            }
            umma_commit(mma_done);
            mbar_wait_drain(mma_done, 0);
        }
    } else {
        // ------------------------------------------------------- epilogue --
        const int lg = warp & 3;
        const int row = lg * 32 + lane;
        int ci = 0;
        bool ok = true;
        for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
            const int bin = u / (a.nchunk * a.mtiles), rem = u % (a.nchunk * a.mtiles);
            const int q = rem / a.mtiles, mt = rem % a.mtiles;
            const int grow = mt * 128 + row;
            for (int c0 = 0; c0 < a.nkb; c0 += kChunkKb, ++ci) {
                const int buf = ci & 1;
                if (!mbar_wait(&acc_full[buf], (uint32_t)((ci >> 1) & 1), abort_flag, a.err, 14)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t tb = tmem + ((uint32_t)(lg * 32) << 16) + buf * 2 * N;
#pragma unroll
                for (int g = 0; g < NG; ++g) {
                    const int col0 = q * N + g * 16;
                    if (col0 >= a.ncol) break;
                    uint32_t re[16], im[16];
                    tmem_ld16(tb + g * 16, re);
                    tmem_ld16(tb + N + g * 16, im);
                    tmem_wait_ld();
                    if (grow < a.nrows) {
                        float2* o = a.out + ((int64_t)bin * a.ncol + col0) * a.ld + grow;
#pragma unroll
                        for (int t = 0; t < 16; ++t) {
                            if (col0 + t < a.ncol) {
                                float* dst = reinterpret_cast<float*>(o + (int64_t)t * a.ld);
                                const float vr = __uint_as_float(re[t]), vi = __uint_as_float(im[t]);
                                if (c0 == 0) *reinterpret_cast<float2*>(dst) = make_float2(vr, vi);
                                else red_add_v2(dst, vr, vi);
                            }
                        }
                    }
                }
                tc_fence_before();
                mbar_arrive(&acc_empty[buf]);
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols));
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

bool map3(CUtensorMap* m, const void* ptr, uint64_t d0, uint64_t d1, uint64_t d2, uint32_t b0,
          uint32_t b1) {
    auto fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[3] = {d0, d1, d2};
    const cuuint64_t str[2] = {d0 * 2, d0 * 2 * d1};
    const cuuint32_t box[3] = {b0, b1, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(ptr), dims, str, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// grouped column planes [groups][ncolp][bins][8]: the box 8 channels x 1 bin x
// ncb columns x 8 groups lands densely (no swizzle) as [group][column][8], the
// K-major core-matrix layout the B descriptor of the kernel describes
bool map4_grouped(CUtensorMap* m, const void* ptr, uint64_t groups, uint64_t bins, uint64_t ncolp,
                  uint32_t ncb) {
    auto fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[4] = {8, bins, ncolp, groups};
    const cuuint64_t str[3] = {16, 16 * bins, 16 * bins * ncolp};
    const cuuint32_t box[4] = {8, 1, ncb, 8};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(ptr), dims, str, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// column chunks of 16 x kNg[j] columns; a chunk is never wider than the planes
constexpr int kNg[3] = {1, 2, 4};

struct CgState {
    CUtensorMap fa[4], aa[4];        // PSF planes in kernel order (two of them without SW)
    CUtensorMap fb[3][4], ab[3][4];  // per chunk width
    CgArgs fwd, adj;
    int sm_count = 0, ncolp = 16, nwidths = 1;
    bool sw = true;
    int* err = nullptr;
};

template <bool ADJ, int NG, bool SW>
cudaError_t launch_width(const CUtensorMap* A, const CUtensorMap* B, CgArgs a, int sm_count,
                         cudaStream_t st) {
    using G = Cg<NG, SW>;
    a.nchunk = (a.ncol + G::N - 1) / G::N;
    const int grid = std::min(a.nbins * a.nchunk * a.mtiles, sm_count);
    k_tc_cgemm<ADJ, NG, SW><<<grid, kThreads, G::kSmemBytes, st>>>(A[0], A[1], A[2], A[3], B[0], B[1],
                                                                   B[2], B[3], a);
    count_launch();
    return cudaGetLastError();
}

template <bool ADJ>
cudaError_t launch(CgState* s, int ncol, cudaStream_t st) {
    if (ncol < 1 || ncol > s->ncolp) return cudaErrorInvalidValue;
    CgArgs a = ADJ ? s->adj : s->fwd;
    a.ncol = ncol;
    // the narrowest chunk that covers all columns, else the widest available
    const int ncg = (ncol + 15) / 16;
    int j = 0;
    while (j + 1 < s->nwidths && kNg[j] < ncg) ++j;
    const CUtensorMap* A = ADJ ? s->aa : s->fa;
    const CUtensorMap* B = ADJ ? s->ab[j] : s->fb[j];
    if (s->sw) {
        switch (kNg[j]) {
            case 1: return launch_width<ADJ, 1, true>(A, B, a, s->sm_count, st);
            case 2: return launch_width<ADJ, 2, true>(A, B, a, s->sm_count, st);
            default: return launch_width<ADJ, 4, true>(A, B, a, s->sm_count, st);
        }
    }
    switch (kNg[j]) {
        case 1: return launch_width<ADJ, 1, false>(A, B, a, s->sm_count, st);
        case 2: return launch_width<ADJ, 2, false>(A, B, a, s->sm_count, st);
        default: return launch_width<ADJ, 4, false>(A, B, a, s->sm_count, st);
    }
}

template <int NG, bool SW>
cudaError_t set_smem() {
    constexpr int bytes = Cg<NG, SW>::kSmemBytes;
    cudaError_t e = cudaFuncSetAttribute(k_tc_cgemm<false, NG, SW>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_tc_cgemm<true, NG, SW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                bytes);
}

}  // namespace

cudaError_t cgemm_init(const CgemmBuffers& b, int sm_count, void** state, std::string* why) {
    CgState* s = new (std::nothrow) CgState();
    if (!s) return cudaErrorMemoryAllocation;
    std::memset(s, 0, sizeof(*s));
    *state = s;
    cudaError_t e = cudaMalloc(&s->err, sizeof(int));
    if (e != cudaSuccess) return e;
    if ((e = cudaMemset(s->err, 0, sizeof(int))) != cudaSuccess) return e;
    s->nwidths = 1;
    while (s->nwidths < 3 && 16 * kNg[s->nwidths] <= b.ncolp) ++s->nwidths;
    s->sw = b.W[1] && b.W[3];
    for (int i = 0; i < 4; ++i) {
        // without the lo planes the kernel's PSF planes are 0 (real hi), 2 (imag hi)
        const __nv_bfloat16* w = s->sw ? b.W[i] : b.W[(i & 1) * 2];
        bool ok = w && map3(&s->fa[i], w, b.Cw, b.S, b.bins, 64, 128) &&
                  map3(&s->aa[i], w, b.Cw, b.S, b.bins, 64, 64);
        for (int j = 0; j < s->nwidths && ok; ++j)
            ok = map4_grouped(&s->fb[j][i], b.X[i], b.Cw / 8, b.bins, b.ncolp, 16 * kNg[j]) &&
                 map4_grouped(&s->ab[j][i], b.Y[i], b.Sw / 8, b.bins, b.ncolp, 16 * kNg[j]);
        if (!ok) {
            if (why) *why = "cuTensorMapEncodeTiled failed for the spectra planes";
            return cudaErrorInvalidValue;
        }
    }
    CgArgs& f = s->fwd;
    f.nbins = b.bins;
    f.ncol = 16;
    f.nchunk = 1;
    f.mtiles = (b.S + 127) / 128;
    f.nkb = (b.Cw + 63) / 64;
    f.nrows = b.S;
    f.ld = b.Sf;
    f.out = b.Yout;
    f.err = s->err;
    CgArgs& g = s->adj;
    g = f;
    g.mtiles = (b.C + 127) / 128;
    g.nkb = (b.Sw + 63) / 64;
    g.nrows = b.C;
    g.ld = b.Cf;
    g.out = b.Xout;
    s->sm_count = sm_count;
    s->ncolp = b.ncolp;
    if (s->sw) {
        if ((e = set_smem<1, true>()) != cudaSuccess) return e;
        if ((e = set_smem<2, true>()) != cudaSuccess) return e;
        return set_smem<4, true>();
    }
    if ((e = set_smem<1, false>()) != cudaSuccess) return e;
    if ((e = set_smem<2, false>()) != cudaSuccess) return e;
    return set_smem<4, false>();
}

cudaError_t cgemm_forward(void* state, int ncol, cudaStream_t st) {
    return launch<false>(static_cast<CgState*>(state), ncol, st);
}

cudaError_t cgemm_adjoint(void* state, int ncol, cudaStream_t st) {
    return launch<true>(static_cast<CgState*>(state), ncol, st);
}

int cgemm_error(void* state) {
    CgState* s = static_cast<CgState*>(state);
    if (!s || !s->err) return 0;
    int h = 0;
    if (cudaMemcpy(&h, s->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
    if (h) cudaMemset(s->err, 0, sizeof(int));
    return h;
}

void cgemm_destroy(void* state) {
    CgState* s = static_cast<CgState*>(state);
    if (!s) return;
    if (s->err) cudaFree(s->err);
    delete s;
}

}  // namespace lfd
