// Split-BF16 complex contractions of the FFT variant on the tcgen05 tensor
// cores (per frequency bin of the overlap-save transforms):
//
//   forward  Yh[bin][t][s] = sum_c       Wf[bin][s][c]  Xh[bin][t][c]
//   adjoint  Xh[bin][t][c] = sum_s  conj(Wf[bin][s][c]) Yh[bin][t][s]
//
// Every complex operand is held as four BF16 planes (real hi, real lo, imag
// hi, imag lo; x = hi + lo). The four data planes of a chunk of n columns are
// the N = 4n columns of one B operand [Xr_hi | Xr_lo | Xi_hi | Xi_lo], so each
// PSF plane takes one MMA per k-step: the real planes of Wf accumulate into P,
// the imaginary ones into Q,
//   P = (Wr_hi + Wr_lo) [Xr_hi | Xr_lo | Xi_hi | Xi_lo],   Q = (Wi_hi + Wi_lo) [ ... ],
// and the epilogue forms
//   forward  re = Wr Xr - Wi Xi = P_r - Q_i,   im = Wr Xi + Wi Xr = P_i + Q_r
//   adjoint  re = Wr Yr + Wi Yi = P_r + Q_i,   im = Wr Yi - Wi Yr = P_i - Q_r
// (P_r: the sum of P's Xr_hi and Xr_lo columns, and so on). With BF16 PSF
// spectra (no lo planes of Wf) only the hi planes take part: the spectra are
// rounded once, the transformed data still carry hi + lo, and the spectra
// stream is 4 bytes per complex value instead of 8. With adaptive lo planes the
// PSF's lo planes are kept only for the (bin, 64-channel block) tiles whose
// largest hi value reaches tau x the largest of all spectra (compact planes
// [slot][S][64], slot 0 all zeros); elsewhere the dropped lo part is below
// 2^-9 tau of the largest value, and the k-block runs the hi MMAs only. One
// block owns 128 output rows (phases s for the forward, channels c for the
// adjoint) by a chunk of 16, 32 or 64 columns (frame x tile) of one bin, so a
// spectra tile is loaded once for up to 64 columns; units are ordered
// bin-major so the blocks working on one bin share its spectra in L2. Its K
// loop streams 64-wide blocks of the PSF planes and the chunk's data planes
// through a TMA ring (3 stages for 16 columns, 2 for wider chunks). The
// accumulators (P and Q of one chunk) alternate between two TMEM buffers (one
// buffer of all 512 columns for 64-column chunks), so the drain of one chunk
// overlaps the next; chains are cut every 64 k-blocks and added into the FP32
// output at L2 (the same rounding control as the direct projections). An MMA
// of N = 16 columns costs about as much of the tensor pipe (its A operand read
// from shared memory) as one of N = 64, so the four data planes side by side
// take a quarter of the instructions of one MMA per plane pair. The spectra
// (all of Wf) are read once per projection while the columns fit one chunk:
// the kernels are bound by HBM bandwidth. Single frames (up to 16 columns)
// take two specialised kernels: the forward's wide units (k_tc_cgemm_wide,
// two bins x both row tiles over a copy of the spectra in unit order) and the
// adjoint with the ratio spectra resident in shared memory
// (k_tc_cgemm_adjr, contiguous unit ranges of equal cost). The forward writes
// its outputs group-major [S/8][ncol][bins][8]; the adjoints write theirs
// [C/8][bins][ncol][8], so that a unit's 16 columns of a channel group are one
// 1 KB run of whole lines.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <random>
#include <vector>

#include "tc_cgemm.h"
#include "tc_ptx.h"

namespace lfd {
namespace {

using namespace tcx;

constexpr int kPlaneA = 128 * 64 * 2;  // 16 KB
constexpr int kThreads = 192;
constexpr int kChunkKb = 64;  // 64 k-blocks x 4 k-steps x 3 passes x 2 = 1536 MMA steps

// PSF spectra planes: MODE_BF16 the two hi planes (two products per term:
// W x_hi + W x_lo); MODE_SPLIT four planes (three products per term);
// MODE_ADAPTIVE the two hi planes plus, for the tiles that keep them, the two
// compact lo planes (three products there, two elsewhere).
constexpr int MODE_BF16 = 0, MODE_SPLIT = 1, MODE_ADAPTIVE = 2;

// Shapes of a unit of NG groups of 16 columns (NG = 1, 2 or 4). The four
// data planes of a chunk are the NB = 4 N columns of one B operand, and each
// PSF plane takes one MMA per k-step into the accumulator P (real part of the
// PSF) or Q (imaginary part), each NB columns wide.
template <int NG, int MODE>
struct Cg {
    static constexpr int N = 16 * NG;                        // columns of a chunk
    static constexpr int NB = 4 * N;                         // MMA N
    static constexpr int NA = MODE == MODE_BF16 ? 2 : 4;     // PSF planes per stage
    static constexpr int kPlaneB = N * 64 * 2;               // one data plane of a stage: 2, 4 or 8 KB
    static constexpr int kStageBytes = NA * kPlaneA + 4 * kPlaneB;
    static constexpr int kStages = (232448 - 1280) / kStageBytes < 6 ? (232448 - 1280) / kStageBytes : 6;
    static constexpr int kSmemBytes = kStages * kStageBytes + 1024 + 256;
    static constexpr int kBufs = 2 * 2 * NB <= 512 ? 2 : 1;  // accumulator buffers of (P, Q)
    static constexpr uint32_t kTmemCols = kBufs * 2 * NB;    // 256 or 512
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
    float2* out;       // forward [ld/8][ncol][bins][8], adjoint [ld/8][bins][ncol][8] (group-major)
    int* err;
    const int* lo_slot;  // adaptive lo planes: [bins][nkbc] compact slot, 0 = dropped
    int nkbc;            // 64-channel blocks of the PSF spectra
    const int64_t* ustart;  // resident-data adjoint: first unit of each block (gridDim.x + 1
                            // entries), or null for equal unit counts
};

template <bool ADJ, int NG, int MODE>
__global__ void __launch_bounds__(kThreads, 1)
k_tc_cgemm(const __grid_constant__ CUtensorMap a0, const __grid_constant__ CUtensorMap a1,
           const __grid_constant__ CUtensorMap a2, const __grid_constant__ CUtensorMap a3,
           const __grid_constant__ CUtensorMap bm, const CgArgs a) {
    using G = Cg<NG, MODE>;
    constexpr int kStages = G::kStages, kStageBytes = G::kStageBytes;
    constexpr int N = G::N, NB = G::NB, NA = G::NA, kBufs = G::kBufs;
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
    volatile int* stage_lo = reinterpret_cast<volatile int*>(tmem_slot + 3);  // [kStages]

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
            int stage = 0, issued = 0;
            uint32_t phase = 0;
            bool ok = true;
            // adaptive lo planes: the compact slots of a k-block's channel block
            // (forward) or of a tile's two 64-channel atoms (adjoint), read one
            // step ahead so that the table lookup overlaps the ring's waits
            const int units_per_bin = a.nchunk * a.mtiles;
            auto unit_slots = [&](int u_, int kb_, int& s0, int& s1) {
                s0 = s1 = 0;
                if (MODE != MODE_ADAPTIVE || u_ >= n_units) return;
                const int bin_ = u_ / units_per_bin, mt_ = (u_ % units_per_bin) % a.mtiles;
                const int* ls = a.lo_slot + (int64_t)bin_ * a.nkbc;
                if (!ADJ) {
                    s0 = ls[kb_];
                } else {
                    s0 = 2 * mt_ < a.nkbc ? ls[2 * mt_] : 0;
                    s1 = 2 * mt_ + 1 < a.nkbc ? ls[2 * mt_ + 1] : 0;
                }
            };
            int nxt0, nxt1;
            unit_slots(blockIdx.x, 0, nxt0, nxt1);
            for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
                const int bin = u / units_per_bin, rem = u % units_per_bin;
                const int q = rem / a.mtiles, mt = rem % a.mtiles;
                int ulo0 = 0, ulo1 = 0;
                if (MODE == MODE_ADAPTIVE && ADJ) {  // per unit; the next unit's now
                    ulo0 = nxt0;
                    ulo1 = nxt1;
                    unit_slots(u + gridDim.x, 0, nxt0, nxt1);
                }
                for (int kb = 0; kb < a.nkb && ok; ++kb) {
                    int lo0 = ulo0, lo1 = ulo1;
                    if (MODE == MODE_ADAPTIVE && !ADJ) {  // per k-block; the next step's now
                        lo0 = nxt0;
                        if (kb + 1 < a.nkb) unit_slots(u, kb + 1, nxt0, nxt1);
                        else unit_slots(u + gridDim.x, 0, nxt0, nxt1);
                    }
                    if (!mbar_wait(&empty[stage], phase ^ 1u, abort_flag, a.err, 11)) {
                        ok = false;
                        break;
                    }
                    const bool lo = MODE == MODE_SPLIT || (MODE == MODE_ADAPTIVE && (lo0 | lo1) != 0);
                    if (MODE == MODE_ADAPTIVE) stage_lo[stage] = lo ? 1 : 0;
                    mbar_expect_tx(&full[stage], lo || MODE == MODE_BF16 ? kStageBytes : kStageBytes - 2 * kPlaneA);
                    const uint32_t sA = sbase + stage * kStageBytes, sB = sA + NA * kPlaneA;
#pragma unroll
                    for (int i = 0; i < NA; ++i) {
                        if (MODE == MODE_ADAPTIVE && (i & 1)) {  // compact lo plane [slot][S][64]
                            if (!lo) continue;
                            if (ADJ) {
                                tma_3d(sA + i * kPlaneA, A[i], 0, kb * 64, lo0, &full[stage]);
                                tma_3d(sA + i * kPlaneA + 8192, A[i], 0, kb * 64, lo1, &full[stage]);
                            } else {
                                tma_3d(sA + i * kPlaneA, A[i], 0, mt * 128, lo0, &full[stage]);
                            }
                        } else if (ADJ) {  // MN-major: two 64-channel atoms of 64 phases
                            tma_3d(sA + i * kPlaneA, A[i], mt * 128, kb * 64, bin, &full[stage]);
                            tma_3d(sA + i * kPlaneA + 8192, A[i], mt * 128 + 64, kb * 64, bin, &full[stage]);
                        } else {
                            tma_3d(sA + i * kPlaneA, A[i], kb * 64, mt * 128, bin, &full[stage]);
                        }
                    }
                    // 8 channels x 1 bin x N columns x (8 groups x 4 planes): [group][plane][column][8]
                    tma_4d(sB, &bm, 0, bin, q * N, kb * 32, &full[stage]);
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
            const uint32_t id = idesc_bf16(128, NB, false, ADJ, false);
            int stage = 0, consumed = 0, ci = 0;
            uint32_t phase = 0;
            bool ok = true;
            for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
                for (int c0 = 0; c0 < a.nkb && ok; c0 += kChunkKb, ++ci) {
                    const int c1 = min(a.nkb, c0 + kChunkKb);
                    const int buf = ci % kBufs;
                    if (ci >= kBufs && !mbar_wait(&acc_empty[buf], (uint32_t)(((ci - kBufs) / kBufs) & 1),
                                                  abort_flag, a.err, 12)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t dP = tmem + buf * 2 * NB, dQ = dP + NB;
                    bool first = true;
                    for (int kb = c0; kb < c1 && ok; ++kb) {
                        if (!mbar_wait(&full[stage], phase, abort_flag, a.err, 13)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t sA = sbase + stage * kStageBytes, sB = sA + NA * kPlaneA;
                        const bool lo = MODE == MODE_SPLIT || (MODE == MODE_ADAPTIVE && stage_lo[stage]);
#pragma unroll
                        for (int ks = 0; ks < 4; ++ks) {
                            // A planes: 0 real hi, 1 real lo, 2 imag hi, 3 imag lo (four
                            // planes), or 0 real hi, 1 imag hi
                            uint64_t ad[NA];
#pragma unroll
                            for (int i = 0; i < NA; ++i)
                                ad[i] = ADJ ? sdesc(sA + i * kPlaneA + ks * 2048, 8192, 1024)
                                            : sdesc(sA + i * kPlaneA + ks * 32, 16, 1024);
                            // B: groups 2ks, 2ks + 1 (4N x 16 B apart), rows plane x N + column
                            const uint64_t bd = sdesc_noswz(sB + ks * 2 * NB * 16, NB * 16, 128);
                            const uint32_t acc0 = (first && ks == 0) ? 0u : 1u;
                            constexpr bool four = NA == 4;
                            umma_bf16(dP, ad[0], bd, id, acc0);            // P += Wr_hi [Xr | Xi]
                            umma_bf16(dQ, ad[four ? 2 : 1], bd, id, acc0); // Q += Wi_hi [Xr | Xi]
                            if (four && lo) {
                                umma_bf16(dP, ad[1], bd, id, 1u);          // P += Wr_lo [Xr | Xi]
                                umma_bf16(dQ, ad[3], bd, id, 1u);          // Q += Wi_lo [Xr | Xi]
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
                const int buf = ci % kBufs;
                if (!mbar_wait(&acc_full[buf], (uint32_t)((ci / kBufs) & 1), abort_flag, a.err, 14)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t tb = tmem + ((uint32_t)(lg * 32) << 16) + buf * 2 * NB;
#pragma unroll
                for (int g = 0; g < NG; ++g) {
                    const int col0 = q * N + g * 16;
                    if (col0 >= a.ncol) break;
                    // P, Q columns plane x N + column: planes 0 real hi, 1 real lo, 2 imag hi, 3 imag lo
                    const uint32_t tP = tb + g * 16, tQ = tP + NB;
                    float re[16], im[16];
                    {
                        uint32_t x0[16], x1[16], x2[16], x3[16];
                        tmem_ld16(tP, x0);
                        tmem_ld16(tP + N, x1);
                        tmem_ld16(tQ + 2 * N, x2);
                        tmem_ld16(tQ + 3 * N, x3);
                        tmem_wait_ld();
#pragma unroll
                        for (int t = 0; t < 16; ++t) {  // forward Wr Xr - Wi Xi, adjoint Wr Yr + Wi Yi
                            const float pr = __uint_as_float(x0[t]) + __uint_as_float(x1[t]);
                            const float qi = __uint_as_float(x2[t]) + __uint_as_float(x3[t]);
                            re[t] = ADJ ? pr + qi : pr - qi;
                        }
                        tmem_ld16(tP + 2 * N, x0);
                        tmem_ld16(tP + 3 * N, x1);
                        tmem_ld16(tQ, x2);
                        tmem_ld16(tQ + N, x3);
                        tmem_wait_ld();
#pragma unroll
                        for (int t = 0; t < 16; ++t) {  // forward Wr Xi + Wi Xr, adjoint Wr Yi - Wi Yr
                            const float pi = __uint_as_float(x0[t]) + __uint_as_float(x1[t]);
                            const float qr = __uint_as_float(x2[t]) + __uint_as_float(x3[t]);
                            im[t] = ADJ ? pi - qr : pi + qr;
                        }
                    }
                    if (grow < a.nrows) {
                        // group-major outputs: forward [ld/8][ncol][bins][8] (the
                        // inverse transform reads a column's bins of 8 rows as one
                        // run), adjoint [ld/8][bins][ncol][8] (a unit's 16 columns
                        // of a group are one 1 KB run, so its writes fill whole
                        // lines; the inverse transform's blocks of one group read
                        // the columns of a bin together)
                        float2* o = ADJ ? a.out + (((int64_t)(grow >> 3) * a.nbins + bin) * a.ncol + col0) * 8 +
                                              (grow & 7)
                                        : a.out + (((int64_t)(grow >> 3) * a.ncol + col0) * a.nbins + bin) * 8 +
                                              (grow & 7);
                        const int64_t ts = ADJ ? 8 : (int64_t)a.nbins * 8;  // float2 between columns
#pragma unroll
                        for (int t = 0; t < 16; ++t) {
                            if (col0 + t < a.ncol) {
                                float* dst = reinterpret_cast<float*>(o + t * ts);
                                if (c0 == 0) *reinterpret_cast<float2*>(dst) = make_float2(re[t], im[t]);
                                else red_add_v2(dst, re[t], im[t]);
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

// Wide forward units (adaptive lo planes, single chunks of up to 16 columns,
// S <= 256). A unit is (bin pair p = bins 2p and 2p + 1, chunk q) and covers
// both row tiles of both bins, so each 32-byte sector of the data planes (8
// channels of two neighbouring bins) is fetched by one unit only, and the data
// of a k-block feeds all four (bin, row tile) accumulator pairs. A k-block is
// 16 channels (one MMA K step). A stage holds per bin the (bin, k-block) group
// of the wide PSF copy, hi and (where the bin's 64-channel block keeps it) lo,
// each one bulk copy of 64 S bytes laid out [row tile][plane][group][rows][8],
// and the bin's four data planes side by side as the N = 64 columns of one B
// operand, [group][plane][column][8] (one TMA box per bin). Each
// PSF part then takes two MMAs per (bin, row tile):
//   P += Wr [Xr_hi | Xr_lo | Xi_hi | Xi_lo],   Q += Wi [Xr_hi | Xr_lo | Xi_hi | Xi_lo]
// (Wr, Wi the hi part, and the lo part where kept), and the epilogue forms
//   re = P[0:16] + P[16:32] - Q[32:48] - Q[48:64],
//   im = P[32:48] + P[48:64] + Q[0:16] + Q[16:32].
// (The lo x lo products of kept tiles are included.) The A descriptors of row
// tile m step over its rows_m rows per channel group; an MMA reads 128 rows,
// and the rows past rows_m (beyond the tile's phases, read from the next piece
// or the group's spare bytes) only reach output rows that are not written.
constexpr int kWideThreads = 192;
constexpr int kWideGroup = 16384;  // bytes reserved per (bin, hi / lo) group: 64 x 256
constexpr int kWideB = 2048;       // B of one bin: 2 groups x 4 planes x 16 columns x 16 B
constexpr int kWideStage = 4 * kWideGroup + 2 * kWideB;  // 68 KB
constexpr int kWideStages = 3;
constexpr int kWideSmem = kWideStages * kWideStage + 1024 + 256;
constexpr int kWideChain = 256;       // k-blocks per accumulation chain
constexpr uint32_t kWideTmem = 512;   // 4 (bin, row tile) x (P, Q) x 64 columns, one buffer
static_assert(kWideSmem <= 232448, "wide stage ring exceeds the shared memory of a block");

struct WideArgs {
    int npairs;         // bin pairs (bins / 2)
    int nchunk;         // chunks of 16 columns
    int ncol;           // output columns of this launch
    int nkb;            // k-blocks of 16 channels per bin
    int S;              // phases (output rows), <= 256
    int mtiles;         // row tiles of 128 (1 or 2)
    int nbins;
    int nkbc;           // 64-channel blocks per bin (lo slot table row length)
    const uint8_t* hi;  // wide hi groups: 64 S bytes per (bin, k-block)
    const uint8_t* lo;  // wide lo groups: 64 S bytes per (slot, k-block of the slot)
    const int* lo_slot; // [bins][nkbc], 0 = dropped
    float2* out;        // [Sf/8][ncol][bins][8] (group-major)
    int* err;
};

__global__ void __launch_bounds__(kWideThreads, 1)
k_tc_cgemm_wide(const __grid_constant__ CUtensorMap bm, const WideArgs a) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t sbase = (raw + 1023u) & ~1023u;
    uint8_t* smem = smem_raw + (sbase - raw);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kWideStages * kWideStage);
    uint64_t* empty = full + kWideStages;
    uint64_t* acc_full = empty + kWideStages;
    uint64_t* acc_empty = acc_full + 1;
    uint64_t* mma_done = acc_empty + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_done + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    volatile int* consumed_ctr = reinterpret_cast<volatile int*>(tmem_slot + 2);
    volatile int* stage_lo = reinterpret_cast<volatile int*>(tmem_slot + 3);  // [kWideStages]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_units = a.npairs * a.nchunk;
    const uint32_t grp = 64u * (uint32_t)a.S;  // bytes of one (bin, k-block) group
    const int rows0 = a.S < 128 ? a.S : 128, rows1 = a.S - rows0;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kWideStages; ++s) {
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
                     "r"(kWideTmem));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ------------------------------------------------- copy producer --
            int stage = 0, issued = 0;
            uint32_t phase = 0;
            bool ok = true;
            // the bins' lo slots of a 64-channel block, read one block ahead so
            // that the table lookup overlaps the ring's waits
            auto slots = [&](int u_, int blk, int& s0, int& s1) {
                s0 = s1 = 0;
                if (u_ >= n_units) return;
                const int* ls = a.lo_slot + (int64_t)(2 * (u_ / a.nchunk)) * a.nkbc + blk;
                s0 = ls[0];
                s1 = ls[a.nkbc];
            };
            int nx0, nx1;
            slots(blockIdx.x, 0, nx0, nx1);
            for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
                const int p = u / a.nchunk, q = u % a.nchunk;
                int sl0 = 0, sl1 = 0;
                for (int kb = 0; kb < a.nkb; ++kb) {
                    if ((kb & 3) == 0) {
                        sl0 = nx0;
                        sl1 = nx1;
                        if (kb + 4 < a.nkb) slots(u, (kb >> 2) + 1, nx0, nx1);
                        else slots(u + gridDim.x, 0, nx0, nx1);
                    }
                    if (!mbar_wait(&empty[stage], phase ^ 1u, abort_flag, a.err, 11)) {
                        ok = false;
                        break;
                    }
                    stage_lo[stage] = (sl0 ? 1 : 0) | (sl1 ? 2 : 0);
                    mbar_expect_tx(&full[stage], 2 * grp + (sl0 ? grp : 0u) + (sl1 ? grp : 0u) + 2 * kWideB);
                    const uint32_t sA = sbase + stage * kWideStage, sB = sA + 4 * kWideGroup;
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        const int bin = 2 * p + j, sl = j ? sl1 : sl0;
                        bulk_g2s(sA + j * kWideGroup, a.hi + ((int64_t)bin * a.nkb + kb) * grp, grp, &full[stage]);
                        if (sl)
                            bulk_g2s(sA + (2 + j) * kWideGroup, a.lo + ((int64_t)sl * 4 + (kb & 3)) * grp, grp,
                                     &full[stage]);
                        // 8 channels x 1 bin x 16 columns x (2 groups x 4 planes)
                        tma_4d(sB + j * kWideB, &bm, 0, bin, q * 16, kb * 8, &full[stage]);
                    }
                    ++issued;
                    if (++stage == kWideStages) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (!ok)
                for (int i = *consumed_ctr; i < issued; ++i)
                    mbar_wait_drain(&full[i % kWideStages], (uint32_t)((i / kWideStages) & 1));
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------------------------------------------- MMA issuer --
            const uint32_t id = idesc_bf16(128, 64, false, false, false);
            int stage = 0, consumed = 0, ci = 0;
            uint32_t phase = 0;
            bool ok = true;
            for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
                for (int c0 = 0; c0 < a.nkb && ok; c0 += kWideChain, ++ci) {
                    const int c1 = min(a.nkb, c0 + kWideChain);
                    if (ci >= 1 && !mbar_wait(acc_empty, (uint32_t)((ci - 1) & 1), abort_flag, a.err, 12)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    for (int kb = c0; kb < c1 && ok; ++kb) {
                        if (!mbar_wait(&full[stage], phase, abort_flag, a.err, 13)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t sA = sbase + stage * kWideStage, sB = sA + 4 * kWideGroup;
                        const int lo = stage_lo[stage];
                        const uint32_t acc0 = kb == c0 ? 0u : 1u;
#pragma unroll
                        for (int j = 0; j < 2; ++j) {
                            // B: 64 rows (plane x 16 + column) of 16 channels; groups 1 KB apart
                            const uint64_t bd = sdesc_noswz(sB + j * kWideB, 1024, 128);
                            const bool jlo = (lo >> j) & 1;
                            for (int m = 0; m < a.mtiles; ++m) {
                                const uint32_t rows = m ? rows1 : rows0, lbo = rows * 16;
                                const uint32_t off = m ? 4u * rows0 * 16 : 0u;
                                const uint32_t hA = sA + j * kWideGroup + off, lA = sA + (2 + j) * kWideGroup + off;
                                const uint32_t dP = tmem + (j * 2 + m) * 128, dQ = dP + 64;
                                umma_bf16(dP, sdesc_noswz(hA, lbo, 128), bd, id, acc0);
                                umma_bf16(dQ, sdesc_noswz(hA + 2 * lbo, lbo, 128), bd, id, acc0);
                                if (jlo) {
                                    umma_bf16(dP, sdesc_noswz(lA, lbo, 128), bd, id, 1u);
                                    umma_bf16(dQ, sdesc_noswz(lA + 2 * lbo, lbo, 128), bd, id, 1u);
                                }
                            }
                        }
                        umma_commit(&empty[stage]);
                        *consumed_ctr = ++consumed;
                        if (++stage == kWideStages) {
                            stage = 0;
                            phase ^= 1u;
                        }
                    }
                    if (ok) umma_commit(acc_full);
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
            const int p = u / a.nchunk, q = u % a.nchunk, col0 = q * 16;
            for (int c0 = 0; c0 < a.nkb; c0 += kWideChain, ++ci) {
                if (!mbar_wait(acc_full, (uint32_t)(ci & 1), abort_flag, a.err, 14)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t tb = tmem + ((uint32_t)(lg * 32) << 16);
                for (int j = 0; j < 2; ++j) {
                    for (int m = 0; m < a.mtiles; ++m) {
                        const uint32_t tP = tb + (j * 2 + m) * 128, tQ = tP + 64;
                        float re[16], im[16];
                        {
                            uint32_t x0[16], x1[16], x2[16], x3[16];
                            tmem_ld16(tP, x0);
                            tmem_ld16(tP + 16, x1);
                            tmem_ld16(tQ + 32, x2);
                            tmem_ld16(tQ + 48, x3);
                            tmem_wait_ld();
#pragma unroll
                            for (int t = 0; t < 16; ++t)
                                re[t] = (__uint_as_float(x0[t]) + __uint_as_float(x1[t])) -
                                        (__uint_as_float(x2[t]) + __uint_as_float(x3[t]));
                            tmem_ld16(tP + 32, x0);
                            tmem_ld16(tP + 48, x1);
                            tmem_ld16(tQ, x2);
                            tmem_ld16(tQ + 16, x3);
                            tmem_wait_ld();
#pragma unroll
                            for (int t = 0; t < 16; ++t)
                                im[t] = (__uint_as_float(x0[t]) + __uint_as_float(x1[t])) +
                                        (__uint_as_float(x2[t]) + __uint_as_float(x3[t]));
                        }
                        const int grow = m * 128 + row;
                        if (grow < a.S) {
                            float2* o = a.out + (((int64_t)(grow >> 3) * a.ncol + col0) * a.nbins + 2 * p + j) * 8 +
                                        (grow & 7);
#pragma unroll
                            for (int t = 0; t < 16; ++t) {
                                if (col0 + t < a.ncol) {
                                    float* dst = reinterpret_cast<float*>(o + (int64_t)t * a.nbins * 8);
                                    if (c0 == 0) *reinterpret_cast<float2*>(dst) = make_float2(re[t], im[t]);
                                    else red_add_v2(dst, re[t], im[t]);
                                }
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
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kWideTmem));
}

// Adjoint units with the data resident (single chunks of up to 16 columns,
// Sw <= 256). The ratio spectra of one bin are 4 k-blocks x 8 KB; a block owns
// a contiguous range of (bin, row tile) units in bin-major order, keeps the
// current bin's data planes in shared memory (loaded once per bin, about 14
// bins per block at the large frame), and streams only the PSF planes through
// its ring. Otherwise as k_tc_cgemm<ADJ = true, NG = 1>. Waits 15 and 16 are
// the data region's (free for reload, loaded).
constexpr int kResB = 4 * 8192;  // resident data: 4 k-blocks x (8 groups x 4 planes x 16 columns x 16 B)
template <int MODE>
struct CgR {
    static constexpr int NA = MODE == MODE_BF16 ? 2 : 4;
    static constexpr int kStageBytes = NA * kPlaneA;
    static constexpr int kStages =
        (232448 - 1280 - kResB) / kStageBytes < 6 ? (232448 - 1280 - kResB) / kStageBytes : 6;
    static constexpr int kSmemBytes = kStages * kStageBytes + kResB + 1024 + 256;
    static_assert(kStages >= 2 && kSmemBytes <= 232448, "stage ring exceeds the shared memory of a block");
};

template <int MODE>
__global__ void __launch_bounds__(kThreads, 1)
k_tc_cgemm_adjr(const __grid_constant__ CUtensorMap a0, const __grid_constant__ CUtensorMap a1,
                const __grid_constant__ CUtensorMap a2, const __grid_constant__ CUtensorMap a3,
                const __grid_constant__ CUtensorMap bm, const CgArgs a) {
    using G = CgR<MODE>;
    constexpr int kStages = G::kStages, kStageBytes = G::kStageBytes, NA = G::NA;
    constexpr int N = 16, NB = 64;
    constexpr uint32_t kTmemCols = 256;  // 2 buffers x (P, Q) x 64 columns
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t sbase = (raw + 1023u) & ~1023u;
    uint8_t* smem = smem_raw + (sbase - raw);
    const uint32_t sBres = sbase + kStages * kStageBytes;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes + kResB);
    uint64_t* empty = full + kStages;
    uint64_t* acc_full = empty + kStages;   // [2]
    uint64_t* acc_empty = acc_full + 2;     // [2]
    uint64_t* b_full = acc_empty + 2;
    uint64_t* b_empty = b_full + 1;
    uint64_t* mma_done = b_empty + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_done + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    volatile int* consumed_ctr = reinterpret_cast<volatile int*>(tmem_slot + 2);
    volatile int* b_seen = reinterpret_cast<volatile int*>(tmem_slot + 3);
    volatile int* stage_lo = reinterpret_cast<volatile int*>(tmem_slot + 4);  // [kStages]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t n_units = (int64_t)a.nbins * a.mtiles;
    const int64_t u0 = a.ustart ? a.ustart[blockIdx.x] : (int64_t)blockIdx.x * n_units / gridDim.x;
    const int64_t u1 = a.ustart ? a.ustart[blockIdx.x + 1] : (int64_t)(blockIdx.x + 1) * n_units / gridDim.x;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 128);
        }
        mbar_init(b_full, 1);
        mbar_init(b_empty, 1);
        mbar_init(mma_done, 1);
        *abort_flag = 0;
        *consumed_ctr = 0;
        *b_seen = 0;
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
            int stage = 0, issued = 0, nb = 0, cur_bin = -1;
            uint32_t phase = 0;
            bool ok = true;
            for (int64_t u = u0; u < u1 && ok; ++u) {
                const int bin = (int)(u / a.mtiles), mt = (int)(u % a.mtiles);
                if (bin != cur_bin) {  // the bin's data planes, once the previous bin's MMAs are done
                    if (nb > 0 && !mbar_wait(b_empty, (uint32_t)((nb - 1) & 1), abort_flag, a.err, 15)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(b_full, a.nkb * 8192);
                    for (int kb = 0; kb < a.nkb; ++kb)  // 8 channels x 1 bin x 16 columns x (8 groups x 4 planes)
                        tma_4d(sBres + kb * 8192, &bm, 0, bin, 0, kb * 32, b_full);
                    ++nb;
                    cur_bin = bin;
                }
                int lo0 = 0, lo1 = 0;  // the tile's two 64-channel atoms
                if (MODE == MODE_ADAPTIVE) {
                    const int* ls = a.lo_slot + (int64_t)bin * a.nkbc;
                    lo0 = 2 * mt < a.nkbc ? ls[2 * mt] : 0;
                    lo1 = 2 * mt + 1 < a.nkbc ? ls[2 * mt + 1] : 0;
                }
                const bool lo = MODE == MODE_SPLIT || (MODE == MODE_ADAPTIVE && (lo0 | lo1) != 0);
                for (int kb = 0; kb < a.nkb && ok; ++kb) {
                    if (!mbar_wait(&empty[stage], phase ^ 1u, abort_flag, a.err, 11)) {
                        ok = false;
                        break;
                    }
                    if (MODE == MODE_ADAPTIVE) stage_lo[stage] = lo ? 1 : 0;
                    mbar_expect_tx(&full[stage], lo || MODE == MODE_BF16 ? kStageBytes : kStageBytes - 2 * kPlaneA);
                    const uint32_t sA = sbase + stage * kStageBytes;
#pragma unroll
                    for (int i = 0; i < NA; ++i) {
                        if (MODE == MODE_ADAPTIVE && (i & 1)) {  // compact lo plane [slot][S][64]
                            if (!lo) continue;
                            tma_3d(sA + i * kPlaneA, A[i], 0, kb * 64, lo0, &full[stage]);
                            tma_3d(sA + i * kPlaneA + 8192, A[i], 0, kb * 64, lo1, &full[stage]);
                        } else {  // MN-major: two 64-channel atoms of 64 phases
                            tma_3d(sA + i * kPlaneA, A[i], mt * 128, kb * 64, bin, &full[stage]);
                            tma_3d(sA + i * kPlaneA + 8192, A[i], mt * 128 + 64, kb * 64, bin, &full[stage]);
                        }
                    }
                    ++issued;
                    if (++stage == kStages) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (!ok) {
                for (int i = *consumed_ctr; i < issued; ++i)
                    mbar_wait_drain(&full[i % kStages], (uint32_t)((i / kStages) & 1));
                if (nb > *b_seen) mbar_wait_drain(b_full, (uint32_t)((nb - 1) & 1));
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------------------------------------------- MMA issuer --
            const uint32_t id = idesc_bf16(128, NB, false, true, false);
            int stage = 0, consumed = 0, ci = 0, nb = 0, cur_bin = -1;
            uint32_t phase = 0;
            bool ok = true;
            for (int64_t u = u0; u < u1 && ok; ++u, ++ci) {
                const int bin = (int)(u / a.mtiles);
                if (bin != cur_bin) {
                    if (!mbar_wait(b_full, (uint32_t)(nb & 1), abort_flag, a.err, 16)) {
                        ok = false;
                        break;
                    }
                    *b_seen = ++nb;
                    cur_bin = bin;
                }
                const int buf = ci & 1;
                if (ci >= 2 &&
                    !mbar_wait(&acc_empty[buf], (uint32_t)(((ci - 2) >> 1) & 1), abort_flag, a.err, 12)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t dP = tmem + buf * 2 * NB, dQ = dP + NB;
                for (int kb = 0; kb < a.nkb && ok; ++kb) {
                    if (!mbar_wait(&full[stage], phase, abort_flag, a.err, 13)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sA = sbase + stage * kStageBytes;
                    const bool lo = MODE == MODE_SPLIT || (MODE == MODE_ADAPTIVE && stage_lo[stage]);
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {
                        uint64_t ad[NA];
#pragma unroll
                        for (int i = 0; i < NA; ++i) ad[i] = sdesc(sA + i * kPlaneA + ks * 2048, 8192, 1024);
                        const uint64_t bd = sdesc_noswz(sBres + kb * 8192 + ks * 2 * NB * 16, NB * 16, 128);
                        const uint32_t acc0 = (kb == 0 && ks == 0) ? 0u : 1u;
                        constexpr bool four = NA == 4;
                        umma_bf16(dP, ad[0], bd, id, acc0);             // P += Wr_hi [Yr | Yi]
                        umma_bf16(dQ, ad[four ? 2 : 1], bd, id, acc0);  // Q += Wi_hi [Yr | Yi]
                        if (four && lo) {
                            umma_bf16(dP, ad[1], bd, id, 1u);
                            umma_bf16(dQ, ad[3], bd, id, 1u);
                        }
                    }
                    umma_commit(&empty[stage]);
                    *consumed_ctr = ++consumed;
                    if (++stage == kStages) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
                if (!ok) break;
                umma_commit(&acc_full[buf]);
                if (u + 1 == u1 || (int)((u + 1) / a.mtiles) != bin) umma_commit(b_empty);  // data free
            }
            umma_commit(mma_done);
            mbar_wait_drain(mma_done, 0);
        }
    } else {
        // ------------------------------------------------------- epilogue --
        const int lg = warp & 3;
        const int row = lg * 32 + lane;
        int ci = 0;
        for (int64_t u = u0; u < u1; ++u, ++ci) {
            const int bin = (int)(u / a.mtiles), mt = (int)(u % a.mtiles);
            const int grow = mt * 128 + row;
            const int buf = ci & 1;
            if (!mbar_wait(&acc_full[buf], (uint32_t)((ci >> 1) & 1), abort_flag, a.err, 14)) break;
            tc_fence_after();
            const uint32_t tP = tmem + ((uint32_t)(lg * 32) << 16) + buf * 2 * NB, tQ = tP + NB;
            float re[16], im[16];
            {
                uint32_t x0[16], x1[16], x2[16], x3[16];
                tmem_ld16(tP, x0);
                tmem_ld16(tP + N, x1);
                tmem_ld16(tQ + 2 * N, x2);
                tmem_ld16(tQ + 3 * N, x3);
                tmem_wait_ld();
#pragma unroll
                for (int t = 0; t < 16; ++t)  // Wr Yr + Wi Yi
                    re[t] = (__uint_as_float(x0[t]) + __uint_as_float(x1[t])) +
                            (__uint_as_float(x2[t]) + __uint_as_float(x3[t]));
                tmem_ld16(tP + 2 * N, x0);
                tmem_ld16(tP + 3 * N, x1);
                tmem_ld16(tQ, x2);
                tmem_ld16(tQ + N, x3);
                tmem_wait_ld();
#pragma unroll
                for (int t = 0; t < 16; ++t)  // Wr Yi - Wi Yr
                    im[t] = (__uint_as_float(x0[t]) + __uint_as_float(x1[t])) -
                            (__uint_as_float(x2[t]) + __uint_as_float(x3[t]));
            }
            if (grow < a.nrows) {  // [ld/8][bins][ncol][8], as k_tc_cgemm<ADJ = true>
                float2* o = a.out + ((int64_t)(grow >> 3) * a.nbins + bin) * a.ncol * 8 + (grow & 7);
#pragma unroll
                for (int t = 0; t < 16; ++t)
                    if (t < a.ncol) o[t * 8] = make_float2(re[t], im[t]);
            }
            tc_fence_before();
            mbar_arrive(&acc_empty[buf]);
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
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

// grouped column planes [rows][ncolp][bins][8] (rows: channel group x 4 +
// plane): the box 8 channels x 1 bin x ncb columns x gbox rows lands densely
// (no swizzle) as [group][plane][column][8], the K-major core-matrix layout of
// the B operands the kernels describe (N = 4 ncb rows: plane x ncb + column)
bool map4_grouped(CUtensorMap* m, const void* ptr, uint64_t groups, uint64_t bins, uint64_t ncolp,
                  uint32_t ncb, uint32_t gbox, bool promote = true) {
    auto fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[4] = {8, bins, ncolp, groups};
    const cuuint64_t str[3] = {16, 16 * bins, 16 * bins * ncolp};
    const cuuint32_t box[4] = {8, 1, ncb, gbox};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(ptr), dims, str, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              promote ? CU_TENSOR_MAP_L2_PROMOTION_L2_256B : CU_TENSOR_MAP_L2_PROMOTION_NONE,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

// Contiguous ranges of about equal cost: units st[k] .. st[k+1]-1 for block k
// of `grid` (st[0] = 0, st[grid] = n), every block at least one unit when
// n >= grid. Each boundary is placed where the running cost first passes
// k / grid of the total, so a range exceeds total / grid by less than the
// largest unit cost.
std::vector<int64_t> balanced_ranges(const std::vector<double>& cost, int grid) {
    const int64_t nu = (int64_t)cost.size();
    std::vector<double> pre((size_t)nu + 1, 0.0);
    for (int64_t u = 0; u < nu; ++u) pre[u + 1] = pre[u] + cost[u];
    std::vector<int64_t> st((size_t)grid + 1, 0);
    int64_t u = 0;
    for (int k = 1; k < grid; ++k) {
        const double target = pre[nu] * k / grid;
        while (u < nu && pre[u + 1] <= target) ++u;
        st[k] = std::min(std::max(st[k - 1] + 1, u), nu - (grid - k));  // no block without units
    }
    st[grid] = nu;
    return st;
}

namespace {

// column chunks of 16 x kNg[j] columns; a chunk is never wider than the planes
constexpr int kNg[3] = {1, 2, 4};

struct CgState {
    CUtensorMap fa[4], aa[4];        // PSF planes in kernel order (see the modes)
    CUtensorMap fb[3], ab[3];        // data planes per chunk width
    CUtensorMap fw;                  // data planes, boxes of 2 groups (wide forward units)
    CUtensorMap ar;                  // ratio planes for the resident-data adjoint (no L2 promotion:
                                     // a block reads a bin's 16-byte pieces once, not its neighbours')
    CgArgs fwd, adj;
    WideArgs wide;
    bool use_wide = false;
    bool use_adjr = false;  // adjoint with resident data for chunks of <= 16 columns
    int sm_count = 0, ncolp = 16, nwidths = 1;
    int mode = MODE_SPLIT;
    int* err = nullptr;
    int64_t* ustart = nullptr;  // cost-balanced unit ranges of the resident-data adjoint
    int ugrid = 0;              // blocks they were made for
};

template <bool ADJ, int NG, int MODE>
cudaError_t launch_width(const CUtensorMap* A, const CUtensorMap* B, CgArgs a, int sm_count,
                         cudaStream_t st) {
    using G = Cg<NG, MODE>;
    a.nchunk = (a.ncol + G::N - 1) / G::N;
    const int grid = std::min(a.nbins * a.nchunk * a.mtiles, sm_count);
    k_tc_cgemm<ADJ, NG, MODE><<<grid, kThreads, G::kSmemBytes, st>>>(A[0], A[1], A[2], A[3], *B, a);
    count_launch();
    return cudaGetLastError();
}

template <bool ADJ, int MODE>
cudaError_t launch_mode(int ng, const CUtensorMap* A, const CUtensorMap* B, const CgArgs& a, int sm_count,
                        cudaStream_t st) {
    switch (ng) {
        case 1: return launch_width<ADJ, 1, MODE>(A, B, a, sm_count, st);
        case 2: return launch_width<ADJ, 2, MODE>(A, B, a, sm_count, st);
        default: return launch_width<ADJ, 4, MODE>(A, B, a, sm_count, st);
    }
}

template <bool ADJ>
cudaError_t launch(CgState* s, int ncol, cudaStream_t st) {
    if (ncol < 1 || ncol > s->ncolp) return cudaErrorInvalidValue;
    if (!ADJ && s->use_wide && ncol <= 16) {  // one chunk: the wide units stream the spectra once
        WideArgs w = s->wide;
        w.ncol = ncol;
        w.nchunk = 1;
        const int grid = std::min(w.npairs * w.nchunk, s->sm_count);
        k_tc_cgemm_wide<<<grid, kWideThreads, kWideSmem, st>>>(s->fw, w);
        count_launch();
        return cudaGetLastError();
    }
    CgArgs a = ADJ ? s->adj : s->fwd;
    a.ncol = ncol;
    if (ADJ && s->use_adjr && ncol <= 16) {
        a.nchunk = 1;
        const int grid = (int)std::min<int64_t>((int64_t)a.nbins * a.mtiles, s->sm_count);
        a.ustart = grid == s->ugrid ? s->ustart : nullptr;
        const CUtensorMap* A = s->aa;
        switch (s->mode) {
            case MODE_BF16:
                k_tc_cgemm_adjr<MODE_BF16><<<grid, kThreads, CgR<MODE_BF16>::kSmemBytes, st>>>(
                    A[0], A[1], A[2], A[3], s->ar, a);
                break;
            case MODE_ADAPTIVE:
                k_tc_cgemm_adjr<MODE_ADAPTIVE><<<grid, kThreads, CgR<MODE_ADAPTIVE>::kSmemBytes, st>>>(
                    A[0], A[1], A[2], A[3], s->ar, a);
                break;
            default:
                k_tc_cgemm_adjr<MODE_SPLIT><<<grid, kThreads, CgR<MODE_SPLIT>::kSmemBytes, st>>>(
                    A[0], A[1], A[2], A[3], s->ar, a);
        }
        count_launch();
        return cudaGetLastError();
    }
    // the narrowest chunk that covers all columns, else the widest available
    const int ncg = (ncol + 15) / 16;
    int j = 0;
    while (j + 1 < s->nwidths && kNg[j] < ncg) ++j;
    const CUtensorMap* A = ADJ ? s->aa : s->fa;
    const CUtensorMap* B = ADJ ? &s->ab[j] : &s->fb[j];
    switch (s->mode) {
        case MODE_BF16: return launch_mode<ADJ, MODE_BF16>(kNg[j], A, B, a, s->sm_count, st);
        case MODE_ADAPTIVE: return launch_mode<ADJ, MODE_ADAPTIVE>(kNg[j], A, B, a, s->sm_count, st);
        default: return launch_mode<ADJ, MODE_SPLIT>(kNg[j], A, B, a, s->sm_count, st);
    }
}

template <int MODE>
cudaError_t set_smem() {
    cudaError_t e = cudaSuccess;
    auto one = [&](auto kern, int bytes) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    };
    one(k_tc_cgemm_adjr<MODE>, CgR<MODE>::kSmemBytes);
    one(k_tc_cgemm<false, 1, MODE>, Cg<1, MODE>::kSmemBytes);
    one(k_tc_cgemm<true, 1, MODE>, Cg<1, MODE>::kSmemBytes);
    one(k_tc_cgemm<false, 2, MODE>, Cg<2, MODE>::kSmemBytes);
    one(k_tc_cgemm<true, 2, MODE>, Cg<2, MODE>::kSmemBytes);
    one(k_tc_cgemm<false, 4, MODE>, Cg<4, MODE>::kSmemBytes);
    one(k_tc_cgemm<true, 4, MODE>, Cg<4, MODE>::kSmemBytes);
    return e;
}

// largest |real| / |imag| hi value of every (bin, 64-channel block) tile of the
// PSF spectra [bins][S][Cw]: one block per tile
__global__ void k_tile_max(const __nv_bfloat16* __restrict__ re, const __nv_bfloat16* __restrict__ im, int S,
                           int Cw, int nkbc, float* __restrict__ tmax) {
    const int bin = blockIdx.x / nkbc, kb = blockIdx.x % nkbc;
    const int c = kb * 64 + (threadIdx.x & 63);
    float m = 0.f;
    if (c < Cw) {
        for (int s = threadIdx.x >> 6; s < S; s += blockDim.x >> 6) {
            const int64_t o = ((int64_t)bin * S + s) * Cw + c;
            m = fmaxf(m, fmaxf(fabsf(__bfloat162float(re[o])), fabsf(__bfloat162float(im[o]))));
        }
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ float wm[32];
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, wm[w]);
        tmax[blockIdx.x] = fmaxf(m, wm[0]);
    }
}

// compact lo planes: tile k of the list (bin, block) goes to slot k + 1
__global__ void k_gather_lo(const __nv_bfloat16* __restrict__ lo, const int2* __restrict__ tiles, int S, int Cw,
                            __nv_bfloat16* __restrict__ dst) {
    const int2 t = tiles[blockIdx.x];  // (bin, block)
    __nv_bfloat16* d = dst + (int64_t)(blockIdx.x + 1) * S * 64;
    for (int e = threadIdx.x; e < S * 64; e += blockDim.x) {
        const int s = e >> 6, c = t.y * 64 + (e & 63);
        d[e] = c < Cw ? lo[((int64_t)t.x * S + s) * Cw + c] : __float2bfloat16(0.f);
    }
}

}  // namespace

cudaError_t cgemm_compact_lo(const CgemmBuffers& b, float tau, cudaStream_t st, LoPlanes* out, int64_t* bytes) {
    *out = LoPlanes{};
    const int nkbc = (b.Cw + 63) / 64;
    const int64_t ntiles = (int64_t)b.bins * nkbc;
    float* dmax = nullptr;
    cudaError_t e = cudaMalloc((void**)&dmax, sizeof(float) * ntiles);
    if (e != cudaSuccess) return e;
    k_tile_max<<<(unsigned)ntiles, 256, 0, st>>>(b.W[0], b.W[2], b.S, b.Cw, nkbc, dmax);
    count_launch();
    std::vector<float> tmax(ntiles);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(tmax.data(), dmax, sizeof(float) * ntiles, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(dmax);
    if (e != cudaSuccess) return e;
    float gmax = 0.f;
    for (float m : tmax) gmax = std::max(gmax, m);
    std::vector<int> slot(ntiles, 0);
    std::vector<int2> keep;
    for (int64_t i = 0; i < ntiles; ++i)
        if (tmax[i] >= tau * gmax) {
            keep.push_back(make_int2((int)(i / nkbc), (int)(i % nkbc)));
            slot[i] = (int)keep.size();
        }
    out->nkbc = nkbc;
    out->tiles = ntiles;
    out->kept = (int64_t)keep.size();
    const size_t plane = (keep.size() + 1) * (size_t)b.S * 64;
    int2* dtiles = nullptr;
    auto alloc = [&](void** p, size_t n) {
        if (injected_alloc_failure()) return cudaErrorMemoryAllocation;
        cudaError_t r = cudaMalloc(p, n);
        if (r == cudaSuccess) *bytes += (int64_t)n;
        return r;
    };
    if ((e = alloc((void**)&out->slot, sizeof(int) * ntiles)) != cudaSuccess) return e;
    if ((e = alloc((void**)&out->lo[0], sizeof(__nv_bfloat16) * plane)) != cudaSuccess) return e;
    if ((e = alloc((void**)&out->lo[1], sizeof(__nv_bfloat16) * plane)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(out->slot, slot.data(), sizeof(int) * ntiles, cudaMemcpyHostToDevice, st)) !=
        cudaSuccess)
        return e;
    for (int q = 0; q < 2 && e == cudaSuccess; ++q)  // slot 0: zeros
        e = cudaMemsetAsync(out->lo[q], 0, sizeof(__nv_bfloat16) * b.S * 64, st);
    if (e == cudaSuccess && !keep.empty()) {
        if ((e = cudaMalloc((void**)&dtiles, sizeof(int2) * keep.size())) != cudaSuccess) return e;
        e = cudaMemcpyAsync(dtiles, keep.data(), sizeof(int2) * keep.size(), cudaMemcpyHostToDevice, st);
        for (int q = 0; q < 2 && e == cudaSuccess; ++q) {
            k_gather_lo<<<(unsigned)keep.size(), 256, 0, st>>>(b.W[2 * q + 1], dtiles, b.S, b.Cw, out->lo[q]);
            count_launch();
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        cudaFree(dtiles);
    }
    return e;
}

namespace {

// byte offset of piece (m, plane, g) inside a (bin, k-block) group of the
// wide layout: tile 0's four pieces of rows0 rows, then tile 1's of rows1
__host__ __device__ __forceinline__ int64_t wide_piece(int m, int plane, int g, int rows0, int rows1) {
    return m == 0 ? (int64_t)(plane * 2 + g) * rows0 * 16
                  : (int64_t)4 * rows0 * 16 + (int64_t)(plane * 2 + g) * rows1 * 16;
}

// one block per (bin, k-block): 16-byte pieces of the hi planes
__global__ void k_wide_hi(const __nv_bfloat16* __restrict__ re, const __nv_bfloat16* __restrict__ im, int S,
                          int Cw, int nkb16, __nv_bfloat16* __restrict__ dst) {
    const int bin = blockIdx.x / nkb16, kb = blockIdx.x % nkb16;
    const int rows0 = S < 128 ? S : 128, rows1 = S - rows0;
    uint8_t* d = reinterpret_cast<uint8_t*>(dst) + (int64_t)blockIdx.x * 64 * S;
    for (int e = threadIdx.x; e < 4 * S; e += blockDim.x) {
        const int s = e % S, pg = e / S, plane = pg >> 1, g = pg & 1;
        const int m = s >> 7, r = s & 127, c = kb * 16 + g * 8;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (c < Cw) v = *reinterpret_cast<const uint4*>((plane ? im : re) + ((int64_t)bin * S + s) * Cw + c);
        *reinterpret_cast<uint4*>(d + wide_piece(m, plane, g, rows0, rows1) + (int64_t)r * 16) = v;
    }
}

// one block per (slot, k-block of the slot's 64 channels): the compact lo planes
__global__ void k_wide_lo(const __nv_bfloat16* __restrict__ re, const __nv_bfloat16* __restrict__ im, int S,
                          __nv_bfloat16* __restrict__ dst) {
    const int slot = 1 + blockIdx.x / 4, q = blockIdx.x % 4;
    const int rows0 = S < 128 ? S : 128, rows1 = S - rows0;
    uint8_t* d = reinterpret_cast<uint8_t*>(dst) + ((int64_t)slot * 4 + q) * 64 * S;
    for (int e = threadIdx.x; e < 4 * S; e += blockDim.x) {
        const int s = e % S, pg = e / S, plane = pg >> 1, g = pg & 1;
        const int m = s >> 7, r = s & 127, c = q * 16 + g * 8;
        const uint4 v = *reinterpret_cast<const uint4*>((plane ? im : re) + ((int64_t)slot * S + s) * 64 + c);
        *reinterpret_cast<uint4*>(d + wide_piece(m, plane, g, rows0, rows1) + (int64_t)r * 16) = v;
    }
}

}  // namespace

cudaError_t cgemm_build_wide(const CgemmBuffers& b, const LoPlanes& lo, cudaStream_t st, WidePlanes* out,
                             int64_t* bytes) {
    *out = WidePlanes{};
    if (b.S > 256 || !b.W[0] || !b.W[2] || !lo.slot || !lo.lo[0] || !lo.lo[1]) return cudaErrorInvalidValue;
    const int nkb16 = (b.Cw + 15) / 16;
    const size_t hi_bytes = (size_t)b.bins * nkb16 * 64 * b.S;
    const size_t lo_bytes = (size_t)(lo.kept + 1) * 4 * 64 * b.S;
    cudaError_t e = injected_alloc_failure() ? cudaErrorMemoryAllocation : cudaMalloc((void**)&out->hi, hi_bytes);
    if (e == cudaSuccess) e = cudaMalloc((void**)&out->lo, lo_bytes);
    if (e != cudaSuccess) {
        cgemm_free_wide(out);
        return e;
    }
    *bytes += (int64_t)(hi_bytes + lo_bytes);
    out->nkb16 = nkb16;
    k_wide_hi<<<(unsigned)((int64_t)b.bins * nkb16), 256, 0, st>>>(b.W[0], b.W[2], b.S, b.Cw, nkb16, out->hi);
    count_launch();
    e = cudaGetLastError();
    if (e == cudaSuccess && lo.kept > 0) {
        k_wide_lo<<<(unsigned)(lo.kept * 4), 256, 0, st>>>(lo.lo[0], lo.lo[1], b.S, out->lo);
        count_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e;
}

void cgemm_free_wide(WidePlanes* p) {
    if (p->hi) cudaFree(p->hi);
    if (p->lo) cudaFree(p->lo);
    *p = WidePlanes{};
}

void cgemm_free_lo(LoPlanes* p) {
    if (p->slot) cudaFree(p->slot);
    if (p->lo[0]) cudaFree(p->lo[0]);
    if (p->lo[1]) cudaFree(p->lo[1]);
    *p = LoPlanes{};
}

cudaError_t cgemm_init(const CgemmBuffers& b, int sm_count, void** state, std::string* why) {
    CgState* s = new (std::nothrow) CgState();
    if (!s) return cudaErrorMemoryAllocation;
    std::memset(s, 0, sizeof(*s));
    *state = s;
    cudaError_t e = cudaMalloc(&s->err, sizeof(int));
    if (e != cudaSuccess) return e;
    if ((e = cudaMemset(s->err, 0, sizeof(int))) != cudaSuccess) return e;
    s->nwidths = 1;
    const int widest = b.max_cols > 0 ? b.max_cols : 64;
    while (s->nwidths < 3 && 16 * kNg[s->nwidths] <= b.ncolp && 16 * kNg[s->nwidths] <= widest) ++s->nwidths;
    s->mode = b.lo.slot ? MODE_ADAPTIVE : (b.W[1] && b.W[3]) ? MODE_SPLIT : MODE_BF16;
    const int nslot = (int)b.lo.kept + 1;
    for (int i = 0; i < 4; ++i) {
        bool ok;
        if (s->mode == MODE_ADAPTIVE && (i & 1)) {  // compact lo planes [slot][S][64]
            ok = map3(&s->fa[i], b.lo.lo[i >> 1], 64, b.S, nslot, 64, 128) &&
                 map3(&s->aa[i], b.lo.lo[i >> 1], 64, b.S, nslot, 64, 64);
        } else {
            // BF16 spectra: the kernel's two PSF planes are 0 (real hi), 2 (imag hi)
            const __nv_bfloat16* w = s->mode == MODE_BF16 ? b.W[(i & 1) * 2] : b.W[i];
            ok = w && map3(&s->fa[i], w, b.Cw, b.S, b.bins, 64, 128) &&
                 map3(&s->aa[i], w, b.Cw, b.S, b.bins, 64, 64);
        }
        if (!ok) {
            if (why) *why = "cuTensorMapEncodeTiled failed for the spectra planes";
            return cudaErrorInvalidValue;
        }
    }
    for (int j = 0; j < s->nwidths; ++j) {  // rows of the data maps: group x 4 + plane
        if (!map4_grouped(&s->fb[j], b.X, 4 * (b.Cw / 8), b.bins, b.ncolp, 16 * kNg[j], 32) ||
            !map4_grouped(&s->ab[j], b.Y, 4 * (b.Sw / 8), b.bins, b.ncolp, 16 * kNg[j], 32)) {
            if (why) *why = "cuTensorMapEncodeTiled failed for the data planes";
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
    f.lo_slot = b.lo.slot;
    f.nkbc = b.lo.nkbc;
    CgArgs& g = s->adj;
    g = f;
    g.mtiles = (b.C + 127) / 128;
    g.nkb = (b.Sw + 63) / 64;
    g.nrows = b.C;
    g.ld = b.Cf;
    g.out = b.Xout;
    s->sm_count = sm_count;
    s->ncolp = b.ncolp;
    s->use_adjr = g.nkb <= kResB / 8192;
    if (s->use_adjr && !map4_grouped(&s->ar, b.Y, 4 * (b.Sw / 8), b.bins, b.ncolp, 16, 32, false)) {
        if (why) *why = "cuTensorMapEncodeTiled failed for the ratio planes";
        return cudaErrorInvalidValue;
    }
    if (s->use_adjr && s->mode == MODE_ADAPTIVE) {
        // Units with lo planes stream twice the PSF bytes of those without, and
        // the lo tiles gather at the low frequencies, i.e. in a few ranges of
        // the bin-major unit order: equal unit counts per block left the blocks
        // holding those ranges running long after the others. Each block gets
        // a contiguous range of about equal cost instead (cost of a unit: its
        // PSF planes, 2 or 4 per k-block, plus its output, about half a plane).
        const int64_t nu = (int64_t)g.nbins * g.mtiles;
        const int grid = (int)std::min<int64_t>(nu, sm_count);
        std::vector<int> slot((size_t)g.nbins * g.nkbc);
        e = cudaMemcpy(slot.data(), g.lo_slot, slot.size() * sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return e;
        std::vector<double> cost((size_t)nu);
        for (int64_t u = 0; u < nu; ++u) {
            const int bin = (int)(u / g.mtiles), mt = (int)(u % g.mtiles);
            const int* ls = slot.data() + (size_t)bin * g.nkbc;
            const bool lo = (2 * mt < g.nkbc && ls[2 * mt] != 0) || (2 * mt + 1 < g.nkbc && ls[2 * mt + 1] != 0);
            cost[u] = (lo ? 4.0 : 2.0) + 0.5;
        }
        const std::vector<int64_t> st = balanced_ranges(cost, grid);
        if ((e = cudaMalloc(&s->ustart, sizeof(int64_t) * (grid + 1))) != cudaSuccess) return e;
        if ((e = cudaMemcpy(s->ustart, st.data(), sizeof(int64_t) * (grid + 1), cudaMemcpyHostToDevice)) !=
            cudaSuccess)
            return e;
        s->ugrid = grid;
    }
    if (s->mode == MODE_ADAPTIVE && b.wide.hi && b.S <= 256 && b.bins % 2 == 0) {
        if (!map4_grouped(&s->fw, b.X, 4 * (b.Cw / 8), b.bins, b.ncolp, 16, 8)) {
            if (why) *why = "cuTensorMapEncodeTiled failed for the wide units' data planes";
            return cudaErrorInvalidValue;
        }
        WideArgs& w = s->wide;
        w.npairs = b.bins / 2;
        w.nchunk = 1;
        w.ncol = 16;
        w.nkb = b.wide.nkb16;
        w.S = b.S;
        w.mtiles = (b.S + 127) / 128;
        w.nbins = b.bins;
        w.nkbc = b.lo.nkbc;
        w.hi = reinterpret_cast<const uint8_t*>(b.wide.hi);
        w.lo = reinterpret_cast<const uint8_t*>(b.wide.lo);
        w.lo_slot = b.lo.slot;
        w.out = b.Yout;
        w.err = s->err;
        cudaError_t e = cudaFuncSetAttribute(k_tc_cgemm_wide, cudaFuncAttributeMaxDynamicSharedMemorySize, kWideSmem);
        if (e != cudaSuccess) return e;
        s->use_wide = true;
    }
    switch (s->mode) {
        case MODE_BF16: return set_smem<MODE_BF16>();
        case MODE_ADAPTIVE: return set_smem<MODE_ADAPTIVE>();
        default: return set_smem<MODE_SPLIT>();
    }
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
    if (s->ustart) cudaFree(s->ustart);
    delete s;
}

}  // namespace lfd

// Host-only check of balanced_ranges on seeded synthetic unit costs shaped
// like the adjoint's (runs of costly units with lo planes among cheaper ones):
// the ranges tile 0 .. n-1 in order, none is empty when n >= grid, and none
// exceeds total / grid by the largest unit cost or more.
extern "C" lfd_status lfd_selftest_balanced_ranges(int seed, int n, int grid) {
    if (n < 1 || grid < 1 || grid > n) return LFD_EINVAL;
    std::mt19937_64 rng((uint64_t)seed);
    std::vector<double> cost((size_t)n);
    double total = 0.0, mx = 0.0;
    int run = 0;
    bool lo = false;
    for (int u = 0; u < n; ++u) {
        if (run == 0) {  // a stretch of units with or without lo planes
            lo = rng() % 3 == 0;
            run = 1 + (int)(rng() % 200);
        }
        --run;
        cost[u] = (lo ? 4.0 : 2.0) + 0.5 + (double)(rng() % 100) * 1e-3;
        total += cost[u];
        mx = std::max(mx, cost[u]);
    }
    const std::vector<int64_t> st = lfd::balanced_ranges(cost, grid);
    if ((int)st.size() != grid + 1 || st[0] != 0 || st[grid] != n) return LFD_EINTERNAL;
    for (int k = 0; k < grid; ++k) {
        if (st[k + 1] <= st[k]) return LFD_EINTERNAL;
        double c = 0.0;
        for (int64_t u = st[k]; u < st[k + 1]; ++u) c += cost[u];
        if (c >= total / grid + mx) return LFD_EINTERNAL;
    }
    return LFD_OK;
}
