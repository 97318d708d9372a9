// Light-field projections as implicit GEMMs on the 5th-generation tensor cores
// (tcgen05, sm_103a): TMA-staged BF16 tiles in shared memory, FP32
// accumulators in tensor memory (TMEM).
//
//   forward   Hv[m][s]      = sum_D sum_c  Vp[m_base + m - off(D)][c] * Wp[D][s][c]
//   backward  HtR[m][(z,t)] = sum_D sum_s  Rp[m_base + m + off(D)][s] * Wp[D][s][(z,t)]
//
// (polyphase form and padded row layout: see lfd_internal.h). A block owns a
// 256-row output tile (two M=128 MMAs, accumulators at TMEM columns 0 and 256)
// and up to 256 output columns. The K loop walks (tap, 64-element block); for
// every step one TMA box of the shifted A rows (256 x 128 B) and one box of
// the tap's weights land in a 3-stage shared-memory ring. The weights are the
// B operand in K-major form for the forward (Wp[D] is [s][c], c contiguous)
// and in MN-major form for the backward (same array, contraction over s). In
// split-BF16 mode each step runs three passes: hi*hi, hi*lo, lo*hi.
//
// TF32 mode (kind::tf32): the operands are FP32 copies rounded to TF32
// (round to nearest, 10-bit mantissa), a k-block is 32 values (the same
// 128 bytes, so tiles, swizzle and descriptors are those of BF16), one pass.
// Both operands are K-major: the backprojection reads a transposed copy of
// the packed PSF, [tap][c][s], instead of the MN-major form.
//
// Warp roles (192 threads): warp 0 issues TMA, warp 1 owns TMEM and issues
// the MMAs (one thread), warps 2-5 drain the accumulators to global memory.
// Blocks are persistent over work units (row tile, column tile, K split); a K
// split writes its own partial output, summed later in a fixed order.
//
// Every wait on an mbarrier is bounded (4 s of %globaltimer). On a timeout the
// block raises a shared abort flag, records an error code in global memory,
// waits (bounded) for its own TMA copies and MMAs still in flight, frees TMEM
// and returns; the host reports LFD_ETIMEDOUT.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "tc_gemm.h"
#include "tc_ptx.h"

namespace lfd {
namespace {

using namespace tcx;

constexpr int kStages = 3;
constexpr int kBM = 256;
constexpr int kBK = 64;                       // bf16 elements per k-block = 128 B (32 for TF32)
constexpr int kABytes = kBM * kBK * 2;        // 32 KB
constexpr int kBBytesMax = 256 * kBK * 2;     // 32 KB
constexpr int kStageBytes = kABytes + kBBytesMax;
constexpr int kThreads = 192;
constexpr int kSmemBytes = kStages * kStageBytes + 1024 + 256;
// The tensor cores add each MMA's result into the FP32 accumulator with a
// rounding that loses about half an ulp per step in one direction, so the
// relative error of a long chain grows linearly with its length (measured:
// ~3e-8 per MMA step). Chains are therefore cut after kChainSteps MMA steps:
// the accumulator is drained and added into the FP32 output in registers
// (round to nearest), and the next chunk starts from zero.
constexpr int kChainSteps = 1536;

struct TcArgs {
    int64_t m_base;
    int Lp, T, h;
    int n_mtiles, n_ntiles, nsplit, n_units;
    int kb_per_tap, kb_total;
    int bn;             // accumulator columns (MMA N)
    int n_valid;        // row length of the destination (Spad or Cpad)
    int passes;         // 1 BF16, 3 split BF16
    int taps;           // T*T
    int tap_inner;      // k-block order: 1 = (block, tap) tap fastest; 0 = (tap, block)
    int chunk_kb;       // k-blocks per accumulation chunk (see below)
    int kvalid;         // contraction entries that are not padding (C or S); MMA
                        // k-steps of 16 that start at or past it are skipped
    uint32_t tx_bytes;  // bytes landing per stage
    float* out;
    int64_t slot_stride;
    int* err;
};

struct Unit {
    int split, ntile, mtile, kb_lo, kb_hi;
};
__device__ __forceinline__ Unit decode(const TcArgs& a, int u) {
    Unit r;
    const int per_split = a.n_mtiles * a.n_ntiles;
    r.split = u / per_split;
    const int rem = u % per_split;
    r.ntile = rem / a.n_mtiles;
    r.mtile = rem % a.n_mtiles;
    r.kb_lo = (int)((int64_t)r.split * a.kb_total / a.nsplit);
    r.kb_hi = (int)((int64_t)(r.split + 1) * a.kb_total / a.nsplit);
    return r;
}

template <bool FWD, bool TF32>
__global__ void __launch_bounds__(kThreads, 1)
k_tc_conv(const __grid_constant__ CUtensorMap mA0, const __grid_constant__ CUtensorMap mA1,
          const __grid_constant__ CUtensorMap mB0, const __grid_constant__ CUtensorMap mB1,
          const TcArgs a) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t sbase = (raw + 1023u) & ~1023u;
    uint8_t* smem = smem_raw + (sbase - raw);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes);
    uint64_t* empty = full + kStages;
    uint64_t* acc_full = empty + kStages;
    uint64_t* acc_empty = acc_full + 1;
    uint64_t* mma_done = acc_empty + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_done + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    volatile int* consumed_ctr = reinterpret_cast<volatile int*>(tmem_slot + 2);

    constexpr int kBKe = TF32 ? 32 : kBK;   // elements per k-block (128 bytes)
    constexpr int kKS = TF32 ? 8 : 16;      // elements per MMA step (32 bytes)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(acc_full, 1);
        mbar_init(acc_empty, 128);
        mbar_init(mma_done, 1);
        *abort_flag = 0;
        *consumed_ctr = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ------------------------------------------------- TMA producer --
            int stage = 0, issued = 0;
            uint32_t phase = 0;
            bool ok = true;
            for (int u = blockIdx.x; u < a.n_units && ok; u += gridDim.x) {
                const Unit w = decode(a, u);
                const int64_t m0 = (int64_t)w.mtile * kBM;
                const int n0 = w.ntile * a.bn;
                for (int kb = w.kb_lo; kb < w.kb_hi && ok; ++kb) {
                    const int tap = a.tap_inner ? kb % a.taps : kb / a.kb_per_tap;
                    const int cb = a.tap_inner ? kb / a.taps : kb % a.kb_per_tap;
                    const int Dy = tap / a.T - a.h, Dx = tap % a.T - a.h;
                    const int64_t off = (int64_t)Dy * a.Lp + Dx;
                    const int row = (int)(a.m_base + m0 + (FWD ? -off : off));
                    for (int p = 0; p < a.passes; ++p) {
                        if (!mbar_wait(&empty[stage], phase ^ 1u, abort_flag, a.err, 1)) {
                            ok = false;
                            break;
                        }
                        mbar_expect_tx(&full[stage], a.tx_bytes);
                        const uint32_t sA = sbase + stage * kStageBytes, sB = sA + kABytes;
                        const CUtensorMap* ma = (p == 2) ? &mA1 : &mA0;
                        const CUtensorMap* mb = (p == 1) ? &mB1 : &mB0;
                        tma_2d(sA, ma, cb * kBKe, row, &full[stage]);
                        if (FWD) {
                            tma_3d(sB, mb, cb * kBKe, 0, tap, &full[stage]);
                        } else if (TF32) {  // K-major [tap][c][s]: bn rows of 32 phases
                            tma_3d(sB, mb, cb * kBKe, n0, tap, &full[stage]);
                        } else {
                            for (int j = 0; j < a.bn / 64; ++j)
                                tma_3d(sB + j * 8192, mb, n0 + j * 64, cb * kBK, tap, &full[stage]);
                        }
                        ++issued;
                        if (++stage == kStages) {
                            stage = 0;
                            phase ^= 1u;
                        }
                    }
                }
            }
            if (!ok) {  // drain our own copies still in flight
                for (int i = *consumed_ctr; i < issued; ++i)
                    mbar_wait_drain(&full[i % kStages], (uint32_t)((i / kStages) & 1));
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------------------------------------------- MMA issuer --
            constexpr bool kBMn = !FWD && !TF32;
            const uint32_t idesc = TF32 ? idesc_tf32(128, a.bn) : idesc_bf16(128, a.bn, kBMn);
            int stage = 0, consumed = 0, ci = 0;
            uint32_t phase = 0;
            bool ok = true;
            for (int u = blockIdx.x; u < a.n_units && ok; u += gridDim.x) {
                const Unit w = decode(a, u);
                for (int c0 = w.kb_lo; c0 < w.kb_hi && ok; c0 += a.chunk_kb, ++ci) {
                    const int c1 = min(w.kb_hi, c0 + a.chunk_kb);
                    if (ci > 0 &&
                        !mbar_wait(acc_empty, (uint32_t)((ci - 1) & 1), abort_flag, a.err, 2)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    bool first = true;
                    for (int kb = c0; kb < c1 && ok; ++kb) {
                        for (int p = 0; p < a.passes; ++p) {
                            if (!mbar_wait(&full[stage], phase, abort_flag, a.err, 3)) {
                                ok = false;
                                break;
                            }
                            tc_fence_after();
                            const uint32_t sA = sbase + stage * kStageBytes, sB = sA + kABytes;
                            const int cb = a.tap_inner ? kb / a.taps : kb % a.kb_per_tap;
                            const int ksteps = min(kBKe / kKS, (a.kvalid - cb * kBKe + kKS - 1) / kKS);
#pragma unroll
                            for (int ks = 0; ks < 4; ++ks) {
                                if (ks >= ksteps) break;
                                const uint64_t bd = (FWD || TF32) ? sdesc(sB + ks * 32, 16, 1024)
                                                                  : sdesc(sB + ks * 2048, 8192, 1024);
#pragma unroll
                                for (int half = 0; half < 2; ++half) {
                                    const uint64_t ad = sdesc(sA + half * 16384 + ks * 32, 16, 1024);
                                    if (TF32)
                                        umma_tf32(tmem + half * 256, ad, bd, idesc,
                                                  (first && ks == 0) ? 0u : 1u);
                                    else
                                        umma_bf16(tmem + half * 256, ad, bd, idesc,
                                                  (first && ks == 0) ? 0u : 1u);
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
                    }
                    if (ok) umma_commit(acc_full);
                }
            }
            // all MMAs issued by this thread complete before TMEM is freed
            umma_commit(mma_done);
            mbar_wait_drain(mma_done, 0);
        }
    } else {
        // ------------------------------------------------------- epilogue --
        const int lg = warp & 3;  // TMEM lane quarter this warp may access
        const int row = lg * 32 + lane;
        int ci = 0;
        bool ok = true;
        for (int u = blockIdx.x; u < a.n_units && ok; u += gridDim.x) {
            const Unit w = decode(a, u);
            float* outp = a.out + (int64_t)w.split * a.slot_stride;
            for (int c0 = w.kb_lo; c0 < w.kb_hi; c0 += a.chunk_kb, ++ci) {
                if (!mbar_wait(acc_full, (uint32_t)(ci & 1), abort_flag, a.err, 4)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                // the first chunk of a unit stores, later chunks add; each
                // thread owns its row, so its adds reach a location in order
                const bool first_chunk = c0 == w.kb_lo;
                for (int half = 0; half < 2; ++half) {
                    const int64_t m = (int64_t)w.mtile * kBM + half * 128 + row;
                    float* orow = outp + m * a.n_valid + w.ntile * a.bn;
                    const int ncols = min(a.bn, a.n_valid - w.ntile * a.bn);
                    const uint32_t tbase = tmem + ((uint32_t)(lg * 32) << 16) + half * 256;
                    for (int cc = 0; cc < a.bn; cc += 32) {
                        uint32_t r0[16], r1[16];
                        tmem_ld16(tbase + cc, r0);
                        if (cc + 16 < a.bn) tmem_ld16(tbase + cc + 16, r1);
                        tmem_wait_ld();
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            if (cc + 4 * q < ncols) {
                                if (first_chunk) st_v4(orow + cc + 4 * q, r0 + 4 * q);
                                else red_add_v4(orow + cc + 4 * q, r0 + 4 * q);
                            }
                        if (cc + 16 < a.bn) {
#pragma unroll
                            for (int q = 0; q < 4; ++q)
                                if (cc + 16 + 4 * q < ncols) {
                                    if (first_chunk) st_v4(orow + cc + 16 + 4 * q, r1 + 4 * q);
                                    else red_add_v4(orow + cc + 16 + 4 * q, r1 + 4 * q);
                                }
                        }
                    }
                }
                tc_fence_before();
                mbar_arrive(acc_empty);
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// ----------------------------------------------------- TF32 operand copies --
// x rounded to TF32 (10-bit mantissa), round to nearest with ties away from
// zero; the low 13 bits of the result are zero
__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__global__ void k_tf32_copy(const float* src, float* dst, int64_t n) {  // src == dst allowed
    const int64_t n4 = n >> 2;
    const float4* s4 = reinterpret_cast<const float4*>(src);
    float4* d4 = reinterpret_cast<float4*>(dst);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n4;
         e += (int64_t)gridDim.x * blockDim.x) {
        const float4 v = s4[e];
        d4[e] = make_float4(to_tf32(v.x), to_tf32(v.y), to_tf32(v.z), to_tf32(v.w));
    }
    for (int64_t e = (n4 << 2) + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x)
        dst[e] = to_tf32(src[e]);
}

// WT[tap][c][s] = tf32(W[tap][s][c]) for s < Spad, c < Cpad, through 32 x 32
// shared-memory tiles (grid x: c tiles, y: s tiles, z: taps)
__global__ void k_tf32_transpose(const float* __restrict__ W, float* __restrict__ WT, int Spad, int Cpad) {
    __shared__ float t[32][33];
    const int64_t tap = blockIdx.z;
    const float* w = W + tap * Spad * (int64_t)Cpad;
    float* wt = WT + tap * Spad * (int64_t)Cpad;
    const int c0 = blockIdx.x * 32, s0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int s = s0 + i, c = c0 + threadIdx.x;
        t[i][threadIdx.x] = (s < Spad && c < Cpad) ? w[(int64_t)s * Cpad + c] : 0.f;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int c = c0 + i, s = s0 + threadIdx.x;
        if (c < Cpad && s < Spad) wt[(int64_t)c * Spad + s] = to_tf32(t[threadIdx.x][i]);
    }
}

cudaError_t launch_tf32_copy(const float* src, float* dst, int64_t n, cudaStream_t st) {
    int64_t b = (n / 4 + 255) / 256;
    b = std::max<int64_t>(1, std::min<int64_t>(b, 152 * 16));
    k_tf32_copy<<<(unsigned)b, 256, 0, st>>>(src, dst, n);
    count_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------------------- host --
struct TcState {
    CUtensorMap fa[2], fb[2];   // forward: A = Vpb hi/lo, B = Wb hi/lo (K-major); TF32: Vpt, W32
    CUtensorMap ba[2], bb[2];   // backward: A = Rpb hi/lo, B = Wb hi/lo (MN-major); TF32: Rpt, WT
    TcArgs fwd, bwd;
    int fwd_grid = 0, bwd_grid = 0;
    bool tf32 = false;
    int* err = nullptr;
};

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

bool make_map(CUtensorMap* m, const void* ptr, int rank, const cuuint64_t* dims,
              const cuuint64_t* strides, const cuuint32_t* box,
              CUtensorMapDataType dt = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16) {
    auto fn = encode_fn();
    if (!fn) return false;
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    return fn(m, dt, rank, const_cast<void*>(ptr), dims, strides, box,
              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// smallest split count whose wave efficiency is within 3% of the best
int pick_split(int64_t base_units, int kb_total, int sm_count, int max_split) {
    double best = 0.0;
    std::vector<double> eff(max_split + 1, 0.0);
    for (int s = 1; s <= max_split; ++s) {
        if (kb_total / s < 2 && s > 1) break;
        const int64_t units = base_units * s;
        const int64_t grid = std::min<int64_t>(units, sm_count);
        const int64_t waves = (units + grid - 1) / grid;
        eff[s] = (double)units / (double)(waves * sm_count);
        best = std::max(best, eff[s]);
    }
    for (int s = 1; s <= max_split; ++s)
        if (eff[s] >= 0.97 * best) return s;
    return 1;
}

int fwd_split_for(const Geo& g, int sm) {
    const int kb_total = (int)(g.taps() * (g.Cpad / kBK));
    return pick_split(g.M_pad / kBM, kb_total, sm, 64);
}
int bwd_ntiles(const Geo& g) { return (g.Cpad + 255) / 256; }
int bwd_bn(const Geo& g) { return g.Cpad >= 256 ? 256 : g.Cpad; }
int bwd_split_for(const Geo& g, int sm) {
    const int kb_total = (int)(g.taps() * ((g.Spad + kBK - 1) / kBK));
    return pick_split((g.M_pad / kBM) * bwd_ntiles(g), kb_total, sm, 16);
}

}  // namespace

bool tc_supported(const Geo& g) { return g.Spad <= 256; }

int tc_forward_parts_for(const Geo& g, int sm_count) { return fwd_split_for(g, sm_count); }
int tc_backward_parts_for(const Geo& g, int sm_count) { return bwd_split_for(g, sm_count); }
int tc_forward_parts(const lfd_ctx* ctx) {
    return ctx->tc ? static_cast<const TcState*>(ctx->tc)->fwd.nsplit : 1;
}
int tc_backward_parts(const lfd_ctx* ctx) {
    return ctx->tc ? static_cast<const TcState*>(ctx->tc)->bwd.nsplit : 1;
}

cudaError_t tc_init(lfd_ctx* ctx) {
    const Geo& g = ctx->g;
    if (!tc_supported(g)) {
        ctx->err = "tensor-core projections need Nnum^2 padded to <= 256 (Nnum <= 15)";
        return cudaErrorNotSupported;
    }
    TcState* s = new (std::nothrow) TcState();
    if (!s) return cudaErrorMemoryAllocation;
    std::memset(s, 0, sizeof(*s));
    ctx->tc = s;
    cudaError_t e = cudaMalloc(&s->err, sizeof(int));
    if (e != cudaSuccess) return e;
    e = cudaMemset(s->err, 0, sizeof(int));
    if (e != cudaSuccess) return e;

    const bool split = ctx->opt.precision == LFD_BF16X3;
    const bool tf32 = s->tf32 = ctx->opt.precision == LFD_TF32;
    const int lo = split ? 1 : 0;
    if (tf32) {
        // operands: the TF32-rounded copies Vpt [rows][Cpad], Rpt [rows][Spad],
        // W32 [taps][Spad][Cpad] (rounded in place) and WT [taps][Cpad][Spad]
        if (!ctx->Vpt || !ctx->Rpt || !ctx->WT || !ctx->W32) {
            ctx->err = "TF32 operand buffers missing";
            return cudaErrorInvalidValue;
        }
        const CUtensorMapDataType F32 = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
        const cuuint32_t bn = (cuuint32_t)bwd_bn(g);
        const cuuint64_t da[2] = {(cuuint64_t)g.Cpad, (cuuint64_t)g.rows};
        const cuuint64_t sa[1] = {(cuuint64_t)g.Cpad * 4};
        const cuuint32_t boxa[2] = {32, 256};
        const cuuint64_t dw[3] = {(cuuint64_t)g.Cpad, (cuuint64_t)g.Spad, (cuuint64_t)g.taps()};
        const cuuint64_t sw[2] = {(cuuint64_t)g.Cpad * 4, (cuuint64_t)g.Cpad * 4 * g.Spad};
        const cuuint32_t boxw[3] = {32, (cuuint32_t)g.Spad, 1};
        const cuuint64_t dr[2] = {(cuuint64_t)g.Spad, (cuuint64_t)g.rows};
        const cuuint64_t sr[1] = {(cuuint64_t)g.Spad * 4};
        const cuuint64_t dt[3] = {(cuuint64_t)g.Spad, (cuuint64_t)g.Cpad, (cuuint64_t)g.taps()};
        const cuuint64_t stt[2] = {(cuuint64_t)g.Spad * 4, (cuuint64_t)g.Spad * 4 * g.Cpad};
        const cuuint32_t boxt[3] = {32, bn, 1};
        if (!make_map(&s->fa[0], ctx->Vpt, 2, da, sa, boxa, F32) ||
            !make_map(&s->fb[0], ctx->W32, 3, dw, sw, boxw, F32) ||
            !make_map(&s->ba[0], ctx->Rpt, 2, dr, sr, boxa, F32) ||
            !make_map(&s->bb[0], ctx->WT, 3, dt, stt, boxt, F32))
            goto fail;
        s->fa[1] = s->fa[0];
        s->fb[1] = s->fb[0];
        s->ba[1] = s->ba[0];
        s->bb[1] = s->bb[0];
        // the PSF operands, once: transposed copy first (from the FP32 values),
        // then the forward copy rounded in place
        const int64_t wcount = g.taps() * g.Spad * (int64_t)g.Cpad;
        dim3 tg((unsigned)((g.Cpad + 31) / 32), (unsigned)((g.Spad + 31) / 32), (unsigned)g.taps());
        k_tf32_transpose<<<tg, dim3(32, 8), 0, 0>>>(ctx->W32, ctx->WT, g.Spad, g.Cpad);
        count_launch();
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        e = launch_tf32_copy(ctx->W32, ctx->W32, wcount, 0);
        if (e != cudaSuccess) return e;
        e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return e;
    }
    // forward A: Vpb [rows][Cpad]; B: Wb [taps][Spad][Cpad]
    for (int b = 0; b < 2 && !tf32; ++b) {
        const int idx = b == 0 ? 0 : lo;
        {
            const cuuint64_t dims[2] = {(cuuint64_t)g.Cpad, (cuuint64_t)g.rows};
            const cuuint64_t str[1] = {(cuuint64_t)g.Cpad * 2};
            const cuuint32_t box[2] = {64, 256};
            if (!make_map(&s->fa[b], ctx->Vpb[idx], 2, dims, str, box)) goto fail;
        }
        {
            const cuuint64_t dims[3] = {(cuuint64_t)g.Cpad, (cuuint64_t)g.Spad, (cuuint64_t)g.taps()};
            const cuuint64_t str[2] = {(cuuint64_t)g.Cpad * 2, (cuuint64_t)g.Cpad * 2 * g.Spad};
            const cuuint32_t boxf[3] = {64, (cuuint32_t)g.Spad, 1};
            const cuuint32_t boxb[3] = {64, 64, 1};
            if (!make_map(&s->fb[b], ctx->Wb[idx], 3, dims, str, boxf)) goto fail;
            if (!make_map(&s->bb[b], ctx->Wb[idx], 3, dims, str, boxb)) goto fail;
        }
        {
            const cuuint64_t dims[2] = {(cuuint64_t)g.Spad, (cuuint64_t)g.rows};
            const cuuint64_t str[1] = {(cuuint64_t)g.Spad * 2};
            const cuuint32_t box[2] = {64, 256};
            if (!make_map(&s->ba[b], ctx->Rpb[idx], 2, dims, str, box)) goto fail;
        }
    }
    {
        TcArgs& f = s->fwd;
        f.m_base = g.m_base;
        f.Lp = g.Lp;
        f.T = g.T;
        f.h = g.h;
        f.n_mtiles = (int)(g.M_pad / kBM);
        f.n_ntiles = 1;
        f.nsplit = fwd_split_for(g, ctx->sm_count);
        f.n_units = f.n_mtiles * f.nsplit;
        // TF32: k-blocks of 32 values, only as many as reach a valid channel
        f.kb_per_tap = tf32 ? (g.C + 31) / 32 : g.Cpad / kBK;
        f.kb_total = (int)(g.taps() * f.kb_per_tap);
        f.bn = g.Spad;
        f.n_valid = g.Spad;
        f.passes = split ? 3 : 1;
        f.taps = (int)g.taps();
        f.tap_inner = 1;
        f.chunk_kb = kChainSteps / (4 * f.passes);
        f.kvalid = g.C;
        f.tx_bytes = (uint32_t)(kABytes + 128 * g.Spad);
        f.out = ctx->Fwd;
        f.slot_stride = g.M_pad * g.Spad;
        f.err = s->err;
        s->fwd_grid = std::min(f.n_units, ctx->sm_count);

        TcArgs& b = s->bwd;
        b = f;
        b.n_ntiles = bwd_ntiles(g);
        b.nsplit = bwd_split_for(g, ctx->sm_count);
        b.n_units = b.n_mtiles * b.n_ntiles * b.nsplit;
        b.kb_per_tap = tf32 ? (g.S + 31) / 32 : (g.Spad + kBK - 1) / kBK;
        b.tap_inner = 0;
        b.kvalid = g.S;
        b.kb_total = (int)(g.taps() * b.kb_per_tap);
        b.bn = bwd_bn(g);
        b.n_valid = g.Cpad;
        b.tx_bytes = (uint32_t)(kABytes + 128 * b.bn);  // bn rows of 128 B (BF16: bn/64 atoms of 8 KB)
        b.out = ctx->Bwd;
        b.slot_stride = g.M_pad * g.Cpad;
        s->bwd_grid = std::min(b.n_units, ctx->sm_count);
    }
    if (tf32) {
        e = cudaFuncSetAttribute(k_tc_conv<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
        if (e != cudaSuccess) return e;
        return cudaFuncSetAttribute(k_tc_conv<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    kSmemBytes);
    }
    e = cudaFuncSetAttribute(k_tc_conv<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_tc_conv<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    return e;
fail:
    ctx->err = "cuTensorMapEncodeTiled failed (or the driver entry point is missing)";
    return cudaErrorInvalidValue;
}

cudaError_t tc_forward(lfd_ctx* ctx, int buf, cudaStream_t st) {
    TcState* s = static_cast<TcState*>(ctx->tc);
    if (!s) return cudaErrorNotReady;
    if (s->tf32) {  // the iterate rounded to TF32 (halo rows and padding stay zero)
        const Geo& g = ctx->g;
        cudaError_t e = launch_tf32_copy(ctx->Vp32[buf], ctx->Vpt, g.rows * g.Cpad, st);
        if (e != cudaSuccess) return e;
        k_tc_conv<true, true><<<s->fwd_grid, kThreads, kSmemBytes, st>>>(s->fa[0], s->fa[1], s->fb[0],
                                                                          s->fb[1], s->fwd);
    } else {
        k_tc_conv<true, false><<<s->fwd_grid, kThreads, kSmemBytes, st>>>(s->fa[0], s->fa[1], s->fb[0],
                                                                           s->fb[1], s->fwd);
    }
    count_launch();
    return cudaGetLastError();
}

cudaError_t tc_backward(lfd_ctx* ctx, cudaStream_t st) {
    TcState* s = static_cast<TcState*>(ctx->tc);
    if (!s) return cudaErrorNotReady;
    if (s->tf32) {  // the ratio image rounded to TF32
        const Geo& g = ctx->g;
        cudaError_t e = launch_tf32_copy(ctx->Rp32, ctx->Rpt, g.rows * g.Spad, st);
        if (e != cudaSuccess) return e;
        k_tc_conv<false, true><<<s->bwd_grid, kThreads, kSmemBytes, st>>>(s->ba[0], s->ba[1], s->bb[0],
                                                                           s->bb[1], s->bwd);
    } else {
        k_tc_conv<false, false><<<s->bwd_grid, kThreads, kSmemBytes, st>>>(s->ba[0], s->ba[1], s->bb[0],
                                                                            s->bb[1], s->bwd);
    }
    count_launch();
    return cudaGetLastError();
}

int tc_error(lfd_ctx* ctx) {
    TcState* s = static_cast<TcState*>(ctx->tc);
    if (!s || !s->err) return 0;
    int h = 0;
    if (cudaMemcpy(&h, s->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
    if (h) cudaMemset(s->err, 0, sizeof(int));
    return h;
}

void tc_destroy(lfd_ctx* ctx) {
    TcState* s = static_cast<TcState*>(ctx->tc);
    if (!s) return;
    if (s->err) cudaFree(s->err);
    delete s;
    ctx->tc = nullptr;
}

}  // namespace lfd
