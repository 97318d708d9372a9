// C ABI of liblfd (include/lfd.h): context set-up, projections, the RL loop
// and the metric, all enqueued on the caller's stream.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <mutex>
#include <vector>

#include "lfd_internal.h"
#include "exact.h"
#include "fft_proj.h"
#include "tc_cgemm.h"
#include "tc_gemm.h"

using namespace lfd;

#define LFD_CK(call)                                                                \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess) {                                                    \
            ctx->err = std::string(#call) + ": " + cudaGetErrorString(e_);          \
            return e_ == cudaErrorMemoryAllocation ? LFD_ENOMEM : LFD_ECUDA;        \
        }                                                                           \
    } while (0)

namespace lfd {

static int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

bool make_geo(int P, int N, int Nz, int H, int W, Geo* g, std::string* why) {
    auto fail = [&](const char* m) {
        if (why) *why = m;
        return false;
    };
    if (N < 1 || (N % 2) == 0) return fail("Nnum must be odd and >= 1");
    if (Nz < 1) return fail("Nz must be >= 1");
    if (P < 1 || (P % 2) == 0) return fail("P must be odd and >= 1");
    if (P % N != 0) return fail("P must be a multiple of Nnum");
    if (H < N || W < N || H % N != 0 || W % N != 0)
        return fail("H and W must be positive multiples of Nnum");
    if ((int64_t)N * N * Nz > (1LL << 24)) return fail("Nnum^2 * Nz too large");
    Geo r{};
    r.N = N;
    r.Nz = Nz;
    r.P = P;
    r.H = H;
    r.W = W;
    r.Ly = H / N;
    r.Lx = W / N;
    r.k = P / N;
    r.h = (r.k + 1) / 2;
    r.T = 2 * r.h + 1;
    r.S = N * N;
    r.Spad = (int)round_up(r.S, 16);
    r.C = Nz * r.S;
    r.Cpad = (int)round_up(r.C, 64);
    r.Lp = r.Lx + r.h;
    r.m_base = r.h + (int64_t)r.h * r.Lp;
    r.M_out = (int64_t)r.Ly * r.Lp;
    r.M_pad = round_up(r.M_out, 256);
    r.rows = r.m_base + r.M_pad + (int64_t)r.h * r.Lp + r.h;
    *g = r;
    return true;
}

std::vector<float2> split_table(const std::vector<double>& t) {
    std::vector<float2> r(t.size());
    for (size_t i = 0; i < t.size(); ++i) {
        const float hi = (float)t[i];
        r[i] = make_float2(hi, (float)(t[i] - (double)hi));
    }
    return r;
}

std::vector<double> dct_table(int n, int Z) {
    // C_k(x; Z) = c(k, Z) cos((2x+1) pi k / (2Z)), c = sqrt(1/Z) for k = 0, sqrt(2/Z) otherwise
    std::vector<double> t((size_t)n * Z);
    const double pi = 3.14159265358979323846;
    for (int k = 0; k < n; ++k) {
        const double ck = k == 0 ? std::sqrt(1.0 / Z) : std::sqrt(2.0 / Z);
        for (int x = 0; x < Z; ++x) t[(size_t)k * Z + x] = ck * std::cos((2.0 * x + 1.0) * pi * k / (2.0 * Z));
    }
    return t;
}

}  // namespace lfd

namespace {

lfd_status rl_step(lfd_ctx* ctx, const float* y, int n, double* entropy_hist, double* flux_hist,
                   cudaStream_t ust);

bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <class T>
lfd_status dalloc(lfd_ctx* ctx, T** p, int64_t count, bool zero) {
    const size_t bytes = (size_t)count * sizeof(T);
    if (injected_alloc_failure()) {
        *p = nullptr;
        ctx->err = "device allocation of " + std::to_string(bytes) + " bytes failed (injected)";
        return LFD_ENOMEM;
    }
    cudaError_t e = cudaMalloc((void**)p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        ctx->err = "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? LFD_ENOMEM : LFD_ECUDA;
    }
    ctx->device_bytes += (int64_t)bytes;
    if (zero) {
        e = cudaMemset(*p, 0, bytes);
        if (e != cudaSuccess) {
            ctx->err = std::string("cudaMemset: ") + cudaGetErrorString(e);
            return LFD_ECUDA;
        }
    }
    return LFD_OK;
}

#define LFD_TRY(x)                       \
    do {                                 \
        lfd_status s_ = (x);             \
        if (s_ != LFD_OK) return s_;     \
    } while (0)

FftBuffers fbufs(const lfd_ctx* ctx) {
    FftBuffers b;
    b.Wf = ctx->Wf;
    b.Xh = ctx->Xh;
    b.Yh = ctx->Yh;
    for (int i = 0; i < 4; ++i) {
        b.Wp[i] = ctx->Wp[i];
        b.Xp[i] = ctx->Xp[i];
        b.Yp[i] = ctx->Yp[i];
    }
    b.cg = ctx->cg;
    if (ctx->fft)
        b.ncolp = (ctx->mf * static_cast<const FftPlan*>(ctx->fft)->ntile + 15) / 16 * 16;
    return b;
}

// direct-variant tensor-core path (BF16, split BF16 or TF32)
bool uses_tc(const lfd_ctx* ctx) {
    return ctx->opt.variant == LFD_DIRECT &&
           (ctx->opt.precision == LFD_BF16 || ctx->opt.precision == LFD_BF16X3 ||
            ctx->opt.precision == LFD_TF32);
}
bool uses_tf32(const lfd_ctx* ctx) { return uses_tc(ctx) && ctx->opt.precision == LFD_TF32; }
bool uses_lo(const lfd_ctx* ctx) { return ctx->opt.precision == LFD_BF16X3; }
// FFT-variant contraction: tensor-core products per term (3 split BF16, 2 BF16
// PSF spectra), 0 for FP32 on the CUDA cores
int fft_products(const lfd_ctx* ctx) {
    return ctx->opt.precision == LFD_BF16X3 ? 3 : ctx->opt.precision == LFD_BF16 ? 2 : 0;
}

// forward projection of Vp32[buf] (and its BF16 copies) into ctx->Fwd
lfd_status run_forward(lfd_ctx* ctx, int buf, cudaStream_t st) {
    const Geo& g = ctx->g;
    if (uses_tc(ctx)) {
        cudaError_t e = tc_forward(ctx, buf, st);
        if (e != cudaSuccess) {
            ctx->err = std::string("tc_forward: ") + cudaGetErrorString(e);
            return LFD_ECUDA;
        }
        return LFD_OK;
    }
    LFD_CK(launch_simt_forward(ctx->Vp32[buf], ctx->W32, g, ctx->fwd_splits, ctx->Fwd, st));
    return LFD_OK;
}

// backprojection of Rp32 (and its BF16 copies) into ctx->Bwd
lfd_status run_backward(lfd_ctx* ctx, cudaStream_t st, bool force_fp32 = false) {
    const Geo& g = ctx->g;
    if (uses_tc(ctx) && !force_fp32) {
        cudaError_t e = tc_backward(ctx, st);
        if (e != cudaSuccess) {
            ctx->err = std::string("tc_backward: ") + cudaGetErrorString(e);
            return LFD_ECUDA;
        }
        return LFD_OK;
    }
    LFD_CK(launch_simt_backward(ctx->Rp32, ctx->W32, g, ctx->bwd_splits, ctx->Bwd, st));
    return LFD_OK;
}

int fwd_parts(const lfd_ctx* ctx) { return uses_tc(ctx) ? tc_forward_parts(ctx) : ctx->fwd_splits; }
int bwd_parts(const lfd_ctx* ctx, bool force_fp32 = false) {
    return (uses_tc(ctx) && !force_fp32) ? tc_backward_parts(ctx) : ctx->bwd_splits;
}

lfd_status ensure_stage(lfd_ctx* ctx, bool vol) {
    const Geo& g = ctx->g;
    if (vol && !ctx->stage_vol)
        return dalloc(ctx, &ctx->stage_vol, (int64_t)ctx->mf * g.Nz * g.H * g.W, false);
    if (!vol && !ctx->stage_img) return dalloc(ctx, &ctx->stage_img, (int64_t)ctx->mf * g.H * g.W, false);
    return LFD_OK;
}

void free_all(lfd_ctx* ctx) {
    void* ptrs[] = {ctx->Vpt, ctx->Rpt, ctx->WT,
                    ctx->W32, ctx->Wb[0], ctx->Wb[1], ctx->Vp32[0], ctx->Vp32[1], ctx->Vpb[0],
                    ctx->Vpb[1], ctx->Rp32, ctx->Rpb[0], ctx->Rpb[1], ctx->Fwd, ctx->Bwd,
                    ctx->invHt1, ctx->ypoly, ctx->mip, ctx->cosW, ctx->cosH, ctx->G, ctx->rowE2,
                    ctx->coef, ctx->flux_part, ctx->hist, ctx->stage_vol, ctx->stage_img,
                    ctx->Wf, ctx->Xh, ctx->Yh, ctx->Vcm[0], ctx->Vcm[1], ctx->Rcm, ctx->Xcm,
                    ctx->invcm, ctx->ycm, ctx->psf_dev, ctx->rimg,
                    ctx->Wp[0], ctx->Wp[1], ctx->Wp[2], ctx->Wp[3], ctx->Xp[0], ctx->Yp[0]};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    exact_plan_destroy(ctx->exact);
    ctx->exact = nullptr;
    if (ctx->lo) {
        cgemm_free_lo(ctx->lo);
        delete ctx->lo;
        ctx->lo = nullptr;
    }
    if (ctx->wide) {
        cgemm_free_wide(ctx->wide);
        delete ctx->wide;
        ctx->wide = nullptr;
    }
    if (ctx->host_pinned) cudaFreeHost(ctx->host_pinned);
    if (ctx->host_hist) cudaFreeHost(ctx->host_hist);
    if (ctx->host_pinned_slots) cudaFreeHost(ctx->host_pinned_slots);
    for (auto& ge : ctx->graph)
        if (ge) cudaGraphExecDestroy(ge);
    if (ctx->ev_in) cudaEventDestroy(ctx->ev_in);
    if (ctx->ev_out) cudaEventDestroy(ctx->ev_out);
    if (ctx->wstream) cudaStreamDestroy(ctx->wstream);
    for (auto& e : ctx->prof.ev)
        if (e) cudaEventDestroy(e);
    ctx->prof.ev.clear();
    tc_destroy(ctx);
    cgemm_destroy(ctx->cg);
    ctx->cg = nullptr;
    delete static_cast<FftPlan*>(ctx->fft);
    ctx->fft = nullptr;
}


}  // namespace

extern "C" {

void lfd_default_options(lfd_options* opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->precision = LFD_FP32;
    opt->eps = 1e-6f;
    opt->dML_um = 150.0;
    opt->Q = 40.0;
    opt->NA = 0.95;
    opt->lambda_um = 0.525;
    opt->XS = 0;
    opt->YS = 0;
    opt->l2_over_region = 1;
    opt->variant = LFD_DIRECT;
    opt->max_frames = 1;
    opt->use_graph = 1;
    opt->fft_size = 0;
    opt->spectra_lo_tau = 0.00390625f;  // 2^-8
}

lfd_status lfd_region_size(int Nnum, int H, int W, double dML_um, double Q, double NA,
                           double lambda_um, int* XS, int* YS) {
    if (!XS || !YS || Nnum < 1 || H < 1 || W < 1 || !(dML_um > 0) || !(Q > 0) || !(NA > 0) ||
        !(lambda_um > 0))
        return LFD_EINVAL;
    // Eq. 7: pixel size in object space; Eq. 11: resolution limit; Eqs. 9-10
    const double P_u = dML_um / (Q * Nnum);
    const double d_psf = 1.22 * lambda_um * Nnum / NA;
    const double xs = P_u * W / d_psf;
    const double ys = P_u * H / d_psf;
    auto clamp = [](double val, int n) {
        double f = std::floor(val);
        const double lo = n < 2 ? n : 2;
        if (!(f >= lo)) f = lo;  // also catches NaN
        if (f > n) f = n;
        return (int)f;
    };
    *XS = clamp(xs, W);
    *YS = clamp(ys, H);
    return LFD_OK;
}

int lfd_predict_stop(const double* E, int n) {
    if (!E || n < 1) return 0;
    for (int k = 1; k < n; ++k)
        if (E[k] < E[k - 1]) return k;
    int best = 0;
    for (int k = 1; k < n; ++k)
        if (E[k] > E[best]) best = k;
    return best + 1;
}

const char* lfd_status_string(lfd_status s) {
    switch (s) {
        case LFD_OK: return "LFD_OK";
        case LFD_EINVAL: return "LFD_EINVAL";
        case LFD_ENOMEM: return "LFD_ENOMEM";
        case LFD_ECUDA: return "LFD_ECUDA";
        case LFD_ENOTREADY: return "LFD_ENOTREADY";
        case LFD_ETIMEDOUT: return "LFD_ETIMEDOUT";
        case LFD_EBUSY: return "LFD_EBUSY";
        case LFD_EINTERNAL: return "LFD_EINTERNAL";
        case LFD_EUNSUPPORTED: return "LFD_EUNSUPPORTED";
        case LFD_ECANCELED: return "LFD_ECANCELED";
    }
    return "unknown";
}

const char* lfd_last_error(const lfd_ctx* ctx) {
    if (!ctx) return "no context";
    return ctx->err.c_str();
}

uint64_t lfd_launch_count(void) { return g_launches.load(); }

lfd_status lfd_create(const float* psf, int P, int Nnum, int Nz, int H, int W,
                      const lfd_options* opt_in, void* cuda_stream, lfd_ctx** out) {
    if (!out) return LFD_EINVAL;
    *out = nullptr;
    if (!psf) return LFD_EINVAL;
    Geo g;
    std::string why;
    if (!make_geo(P, Nnum, Nz, H, W, &g, &why)) return LFD_EINVAL;
    lfd_options opt;
    if (opt_in) opt = *opt_in; else lfd_default_options(&opt);
    if (opt.precision < LFD_FP32 || opt.precision > LFD_BF16X3) return LFD_EINVAL;
    if (!(opt.eps >= 0.f)) return LFD_EINVAL;
    if (opt.variant != LFD_DIRECT && opt.variant != LFD_FFT) return LFD_EINVAL;
    if (opt.max_frames < 1 || opt.max_frames > 4096) return LFD_EINVAL;
    if (opt.fft_size != 0 && opt.fft_size != 32 && opt.fft_size != 64) return LFD_EINVAL;
    if (!(opt.spectra_lo_tau >= 0.f && opt.spectra_lo_tau < 1.f)) return LFD_EINVAL;
    if (opt.contraction_cols != 0 && opt.contraction_cols != 16 && opt.contraction_cols != 32 &&
        opt.contraction_cols != 64)
        return LFD_EINVAL;
    if (opt.max_frames > 1 && opt.variant != LFD_FFT) return LFD_EUNSUPPORTED;
    if (opt.precision == LFD_TF32 && opt.variant != LFD_DIRECT) return LFD_EUNSUPPORTED;
    int XS = opt.XS, YS = opt.YS;
    if (XS <= 0 || YS <= 0) {
        if (lfd_region_size(Nnum, H, W, opt.dML_um, opt.Q, opt.NA, opt.lambda_um, &XS, &YS) != LFD_OK)
            return LFD_EINVAL;
    }
    if (XS > W || YS > H) return LFD_EINVAL;

    lfd_ctx* ctx = new (std::nothrow) lfd_ctx();
    if (!ctx) return LFD_ENOMEM;
    ctx->g = g;
    ctx->opt = opt;
    ctx->XS = XS;
    ctx->YS = YS;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    auto bail = [&](lfd_status s) {
        std::fprintf(stderr, "lfd_create: %s\n", ctx->err.c_str());
        free_all(ctx);
        delete ctx;
        return s;
    };
#define CREATE_CK(call)                                                          \
    do {                                                                         \
        cudaError_t e_ = (call);                                                 \
        if (e_ != cudaSuccess) {                                                 \
            ctx->err = std::string(#call) + ": " + cudaGetErrorString(e_);       \
            return bail(e_ == cudaErrorMemoryAllocation ? LFD_ENOMEM : LFD_ECUDA); \
        }                                                                        \
    } while (0)
#define CREATE_TRY(x)                     \
    do {                                  \
        lfd_status s_ = (x);              \
        if (s_ != LFD_OK) return bail(s_); \
    } while (0)

    CREATE_CK(cudaGetDevice(&ctx->device));
    CREATE_CK(cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, ctx->device));
    if (uses_tc(ctx)) {
        int major = 0, minor = 0;
        CREATE_CK(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, ctx->device));
        CREATE_CK(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, ctx->device));
        if (major != 10) {
            ctx->err = "tensor-core precisions need an sm_10x (Blackwell) device";
            return bail(LFD_EUNSUPPORTED);
        }
        if (!tc_supported(g)) {
            ctx->err = "tensor-core precisions support Nnum <= 15";
            return bail(LFD_EUNSUPPORTED);
        }
    }

    const bool fft = ctx->opt.variant == LFD_FFT;
    FftPlan fplan{};
    if (fft) {
        if (!fft_plan_for(g, &fplan, ctx->opt.fft_size, ctx->opt.max_frames, fft_products(ctx))) {
            ctx->err = "no FFT tiling fits this geometry (at most 64 tiles, Nnum <= 15)";
            return bail(LFD_EUNSUPPORTED);
        }
        FftPlan* hp = new (std::nothrow) FftPlan(fplan);
        if (!hp) return bail(LFD_ENOMEM);
        ctx->fft = hp;
    }
    ctx->fwd_splits = simt_fwd_splits(g, ctx->sm_count);
    ctx->bwd_splits = simt_bwd_splits(g, ctx->sm_count);
    const int64_t wcount = g.taps() * g.Spad * (int64_t)g.Cpad;
    CREATE_TRY(dalloc(ctx, &ctx->W32, wcount, false));
    const int64_t L2 = (int64_t)g.Ly * g.Lx;
    const int mf = ctx->mf = fft ? ctx->opt.max_frames : 1;
    if (fft) {
        const int ncol = mf * fplan.ntile, ncolp = (ncol + 15) / 16 * 16;
        if (fft_products(ctx)) {
            for (int i = 0; i < 4; ++i)
                if (fft_products(ctx) == 3 || i % 2 == 0)  // BF16 spectra: hi planes only
                    CREATE_TRY(dalloc(ctx, &ctx->Wp[i], (int64_t)fplan.bins * g.S * fplan.Cw, false));
            // the four data planes of each 8-channel group side by side (one block)
            CREATE_TRY(dalloc(ctx, &ctx->Xp[0], 4 * (int64_t)fplan.bins * ncolp * fplan.Cw, true));
            CREATE_TRY(dalloc(ctx, &ctx->Yp[0], 4 * (int64_t)fplan.bins * ncolp * fplan.Sw, true));
            for (int i = 1; i < 4; ++i) {
                ctx->Xp[i] = ctx->Xp[0] + (int64_t)i * ncolp * fplan.bins * 8;
                ctx->Yp[i] = ctx->Yp[0] + (int64_t)i * ncolp * fplan.bins * 8;
            }
        } else {
            CREATE_TRY(dalloc(ctx, &ctx->Wf, (int64_t)fplan.bins * g.S * fplan.Cf, false));
        }
        CREATE_TRY(dalloc(ctx, &ctx->Xh, (int64_t)fplan.bins * ncol * fplan.Cf, true));
        CREATE_TRY(dalloc(ctx, &ctx->Yh, (int64_t)fplan.bins * ncol * fplan.Sf, true));
        for (int b = 0; b < 2; ++b) CREATE_TRY(dalloc(ctx, &ctx->Vcm[b], (int64_t)mf * g.C * L2, true));
        CREATE_TRY(dalloc(ctx, &ctx->Rcm, (int64_t)mf * g.S * L2, true));
        CREATE_TRY(dalloc(ctx, &ctx->Xcm, (int64_t)mf * g.C * L2, true));
        CREATE_TRY(dalloc(ctx, &ctx->invcm, (int64_t)g.C * L2, true));
        CREATE_TRY(dalloc(ctx, &ctx->ycm, (int64_t)mf * g.S * L2, true));
        CREATE_TRY(dalloc(ctx, &ctx->rimg, (int64_t)mf * g.H * g.W, true));
        CREATE_TRY(dalloc(ctx, &ctx->psf_dev, (int64_t)Nz * Nnum * Nnum * P * P, false));
        ctx->nflux = update_cm_blocks(g);
    } else {
        // Hv partials serve both the SIMT path and the tensor-core path
        const int fparts = std::max(ctx->fwd_splits, uses_tc(ctx) ? tc_forward_parts_for(g, ctx->sm_count) : 1);
        const int bparts = std::max(ctx->bwd_splits, uses_tc(ctx) ? tc_backward_parts_for(g, ctx->sm_count) : 1);
        for (int b = 0; b < 2; ++b) CREATE_TRY(dalloc(ctx, &ctx->Vp32[b], g.rows * g.Cpad, true));
        CREATE_TRY(dalloc(ctx, &ctx->Rp32, g.rows * g.Spad, true));
        CREATE_TRY(dalloc(ctx, &ctx->Fwd, (int64_t)fparts * g.M_pad * g.Spad, true));
        CREATE_TRY(dalloc(ctx, &ctx->Bwd, (int64_t)bparts * g.M_pad * g.Cpad, true));
        CREATE_TRY(dalloc(ctx, &ctx->invHt1, g.M_pad * g.Cpad, true));
        CREATE_TRY(dalloc(ctx, &ctx->ypoly, g.M_pad * g.Spad, true));
        if (uses_tf32(ctx)) {
            CREATE_TRY(dalloc(ctx, &ctx->WT, wcount, false));
            CREATE_TRY(dalloc(ctx, &ctx->Vpt, g.rows * g.Cpad, true));
            CREATE_TRY(dalloc(ctx, &ctx->Rpt, g.rows * g.Spad, true));
        } else if (uses_tc(ctx)) {
            const int nb = uses_lo(ctx) ? 2 : 1;
            for (int b = 0; b < nb; ++b) {
                CREATE_TRY(dalloc(ctx, &ctx->Wb[b], wcount, false));
                CREATE_TRY(dalloc(ctx, &ctx->Vpb[b], g.rows * g.Cpad, true));
                CREATE_TRY(dalloc(ctx, &ctx->Rpb[b], g.rows * g.Spad, true));
            }
        }
        ctx->nflux = g.Ly * g.Lx;
    }
    CREATE_TRY(dalloc(ctx, &ctx->mip, (int64_t)mf * g.H * g.W, true));
    CREATE_TRY(dalloc(ctx, &ctx->cosW, (int64_t)XS * g.W, false));
    CREATE_TRY(dalloc(ctx, &ctx->cosH, (int64_t)YS * g.H, false));
    CREATE_TRY(dalloc(ctx, &ctx->G, (int64_t)mf * g.H * XS, true));
    CREATE_TRY(dalloc(ctx, &ctx->rowE2, (int64_t)mf * g.H, true));
    CREATE_TRY(dalloc(ctx, &ctx->coef, (int64_t)mf * (XS * YS + kMetricScratch), true));
    CREATE_TRY(dalloc(ctx, &ctx->flux_part, (int64_t)mf * std::max<int64_t>(ctx->nflux, L2), true));
    CREATE_TRY(dalloc(ctx, &ctx->hist, 2LL * mf, true));
    CREATE_CK(cudaMallocHost((void**)&ctx->host_pinned, 4 * sizeof(double)));
    CREATE_CK(cudaMallocHost((void**)&ctx->host_pinned_slots, 2 * sizeof(double) * mf));
    CREATE_CK(cudaStreamCreateWithFlags(&ctx->wstream, cudaStreamNonBlocking));
    CREATE_CK(cudaEventCreateWithFlags(&ctx->ev_in, cudaEventDisableTiming));
    CREATE_CK(cudaEventCreateWithFlags(&ctx->ev_out, cudaEventDisableTiming));

    // PSF to the device (a device pointer is read in place)
    const int64_t psf_count = (int64_t)Nz * Nnum * Nnum * P * P;
    const float* psf_dev = psf;
    float* psf_tmp = nullptr;
    if (!is_device_ptr(psf)) {
        CREATE_CK(cudaMalloc((void**)&psf_tmp, (size_t)psf_count * sizeof(float)));
        cudaError_t e = cudaMemcpyAsync(psf_tmp, psf, (size_t)psf_count * sizeof(float),
                                        cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) {
            cudaFree(psf_tmp);
            CREATE_CK(e);
        }
        psf_dev = psf_tmp;
    }
    cudaError_t e = launch_repack_psf(psf_dev, g, ctx->W32, ctx->Wb[0], ctx->Wb[1], st);
    if (e == cudaSuccess && ctx->psf_dev)
        e = cudaMemcpyAsync(ctx->psf_dev, psf_dev, (size_t)psf_count * sizeof(float),
                            cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (psf_tmp) cudaFree(psf_tmp);
    CREATE_CK(e);

    if (fft) {
        // PSF spectra, then H^T 1 by the FFT backprojection of ones
        CREATE_CK(fft_init(fplan, g, ctx->W32, fbufs(ctx), st));
        if (fft_products(ctx)) {
            int major = 0;
            CREATE_CK(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, ctx->device));
            if (major != 10) {
                ctx->err = "the tensor-core FFT contraction needs an sm_10x (Blackwell) device";
                return bail(LFD_EUNSUPPORTED);
            }
            CgemmBuffers cb{};
            cb.bins = fplan.bins;
            cb.ntile = fplan.ntile;
            cb.ncolp = (ctx->mf * fplan.ntile + 15) / 16 * 16;
            cb.max_cols = ctx->opt.contraction_cols;
            cb.S = g.S;
            cb.C = g.C;
            cb.Sw = fplan.Sw;
            cb.Cw = fplan.Cw;
            cb.Sf = fplan.Sf;
            cb.Cf = fplan.Cf;
            for (int i = 0; i < 4; ++i) cb.W[i] = ctx->Wp[i];
            cb.X = ctx->Xp[0];
            cb.Y = ctx->Yp[0];
            cb.Yout = ctx->Yh;
            cb.Xout = ctx->Xh;
            const int64_t plane_bytes = (int64_t)fplan.bins * g.S * fplan.Cw * (int64_t)sizeof(__nv_bfloat16);
            ctx->spectra_bytes = plane_bytes * (fft_products(ctx) == 3 ? 4 : 2);
            if (fft_products(ctx) == 3 && ctx->opt.spectra_lo_tau > 0.f) {
                // adaptive lo planes: keep the tiles that matter, free the full lo planes
                ctx->lo = new (std::nothrow) LoPlanes();
                if (!ctx->lo) return bail(LFD_ENOMEM);
                CREATE_CK(cgemm_compact_lo(cb, ctx->opt.spectra_lo_tau, st, ctx->lo, &ctx->device_bytes));
                for (int i : {1, 3}) {
                    cudaFree(ctx->Wp[i]);
                    ctx->Wp[i] = nullptr;
                    cb.W[i] = nullptr;
                    ctx->device_bytes -= plane_bytes;
                }
                cb.lo = *ctx->lo;
                ctx->spectra_bytes = plane_bytes * 2 + 2 * (ctx->lo->kept + 1) * (int64_t)g.S * 64 *
                                                           (int64_t)sizeof(__nv_bfloat16);
                if (ctx->mf == 1 && fplan.ntile <= 16 && g.S <= 256) {
                    // single frames: the forward's wide units read their own copy
                    // of the spectra (the same bytes per projection)
                    ctx->wide = new (std::nothrow) WidePlanes();
                    if (!ctx->wide) return bail(LFD_ENOMEM);
                    CREATE_CK(cgemm_build_wide(cb, *ctx->lo, st, ctx->wide, &ctx->device_bytes));
                    cb.wide = *ctx->wide;
                }
            }
            std::string why2;
            cudaError_t ce = cgemm_init(cb, ctx->sm_count, &ctx->cg, &why2);
            if (ce != cudaSuccess) {
                ctx->err = "cgemm_init: " + (why2.empty() ? std::string(cudaGetErrorString(ce)) : why2);
                return bail(LFD_ECUDA);
            }
        }
        CREATE_CK(launch_fill_cm(ctx->Rcm, (int64_t)g.S * L2, 1.0f, st));
        CREATE_CK(fft_backward(fplan, g, fbufs(ctx), 1, ctx->Rcm, ctx->Xcm, nullptr, st, nullptr));
        // Voxels whose sensitivity H^T 1 is below kLowSensitivity of the largest
        // are dominated by the transforms' absolute error floor (~1e-7 of a
        // tile's largest value); list them once and backproject them exactly,
        // here for H^T 1 and in every iteration for H^T r.
        {
            const int64_t nvox = (int64_t)g.C * L2;
            std::vector<float> h(nvox);
            CREATE_CK(cudaMemcpyAsync(h.data(), ctx->Xcm, nvox * sizeof(float), cudaMemcpyDeviceToHost, st));
            CREATE_CK(cudaStreamSynchronize(st));
            float mx = 0.f;
            for (float x : h) mx = x > mx ? x : mx;
            const float thr = kLowSensitivity * mx;
            std::vector<int64_t> low;
            for (int64_t i = 0; i < nvox; ++i)
                if (!(h[i] >= thr)) low.push_back(i);
            ctx->n_low = (int64_t)low.size();
            if (ctx->n_low > 0) {
                std::string why2;
                const cudaError_t pe = exact_plan_create(low.data(), ctx->n_low, g, ctx->psf_dev, mf, st,
                                                         &ctx->exact, &ctx->device_bytes, &why2);
                if (pe != cudaSuccess) {
                    ctx->err = why2;
                    return bail(pe == cudaErrorMemoryAllocation ? LFD_ENOMEM : LFD_ECUDA);
                }
                CREATE_TRY(ensure_stage(ctx, false));
                CREATE_CK(launch_fill(ctx->stage_img, (int64_t)g.H * g.W, 1.0f, st));
                CREATE_CK(exact_bwd(ctx->exact, 1, ctx->stage_img, ctx->Xcm, st));
            }
        }
        CREATE_CK(launch_inv_cm(ctx->Xcm, (int64_t)g.C * L2, ctx->invcm, st));
        CREATE_CK(cudaStreamSynchronize(st));
        cudaFree(ctx->W32);  // the FFT variant reads only the spectra
        ctx->device_bytes -= wcount * (int64_t)sizeof(float);
        ctx->W32 = nullptr;
    } else {
        // H^T 1 (FP32 path) and its reciprocal
        CREATE_TRY(ensure_stage(ctx, false));
        CREATE_CK(launch_fill(ctx->stage_img, (int64_t)g.H * g.W, 1.0f, st));
        CREATE_CK(launch_poly_image(ctx->stage_img, g, ctx->Rp32, g.m_base, nullptr, nullptr, st));
        CREATE_TRY(run_backward(ctx, st, /*force_fp32=*/true));
        CREATE_CK(launch_inv_ht1(ctx->Bwd, ctx->bwd_splits, g, ctx->invHt1, st));
    }

    // metric tables (Eqs. 2-4), FP64 on the host
    {
        const std::vector<float2> tw = split_table(dct_table(XS, g.W));
        const std::vector<double> th = dct_table(YS, g.H);
        CREATE_CK(cudaMemcpyAsync(ctx->cosW, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice, st));
        CREATE_CK(cudaMemcpyAsync(ctx->cosH, th.data(), th.size() * sizeof(double), cudaMemcpyHostToDevice, st));
        CREATE_CK(cudaStreamSynchronize(st));
    }
    if (uses_tc(ctx)) {
        cudaError_t te = tc_init(ctx);
        if (te != cudaSuccess) {
            if (ctx->err.empty()) ctx->err = std::string("tc_init: ") + cudaGetErrorString(te);
            return bail(LFD_ECUDA);
        }
    }
    *out = ctx;
    return LFD_OK;
#undef CREATE_CK
#undef CREATE_TRY
}

void lfd_destroy(lfd_ctx* ctx) {
    if (!ctx) return;
    cudaDeviceSynchronize();
    free_all(ctx);
    delete ctx;
}

lfd_status lfd_get_geometry(const lfd_ctx* ctx, int* XS, int* YS, int* taps, int* precision,
                            int64_t* device_bytes) {
    if (!ctx) return LFD_EINVAL;
    if (XS) *XS = ctx->XS;
    if (YS) *YS = ctx->YS;
    if (taps) *taps = ctx->g.T;
    if (precision) *precision = ctx->opt.precision;
    if (device_bytes) *device_bytes = ctx->device_bytes;
    return LFD_OK;
}

lfd_status lfd_get_fft_plan(const lfd_ctx* ctx, int* F, int* B, int* tiles, int* bins) {
    if (!ctx) return LFD_EINVAL;
    const FftPlan* fp = static_cast<const FftPlan*>(ctx->fft);
    if (F) *F = fp ? fp->F : 0;
    if (B) *B = fp ? fp->B : 0;
    if (tiles) *tiles = fp ? fp->ntile : 0;
    if (bins) *bins = fp ? fp->bins : 0;
    return LFD_OK;
}

lfd_status lfd_get_exact_plan(const lfd_ctx* ctx, int64_t* n_low, int64_t* in_runs, int64_t* runs,
                              int64_t* single) {
    if (!ctx) return LFD_EINVAL;
    if (n_low) *n_low = ctx->exact ? ctx->n_low : 0;
    exact_plan_counts(ctx->exact, in_runs, runs, single);
    return LFD_OK;
}

lfd_status lfd_get_spectra(const lfd_ctx* ctx, int64_t* bytes, int64_t* lo_tiles_kept, int64_t* lo_tiles) {
    if (!ctx) return LFD_EINVAL;
    const FftPlan* fp = static_cast<const FftPlan*>(ctx->fft);
    const bool tc = fp && ctx->cg;
    const int64_t tiles = fp ? (int64_t)fp->bins * ((fp->Cw + 63) / 64) : 0;
    if (bytes) *bytes = tc ? ctx->spectra_bytes : 0;
    if (lo_tiles) *lo_tiles = tc ? tiles : 0;
    if (lo_tiles_kept)
        *lo_tiles_kept = !tc ? 0 : ctx->lo ? ctx->lo->kept : fft_products(ctx) == 3 ? tiles : 0;
    return LFD_OK;
}

lfd_status lfd_forward(lfd_ctx* ctx, const float* v, float* y_out, void* cuda_stream) {
    if (!ctx) return LFD_EINVAL;
    if (!v || !y_out) {
        ctx->err = "NULL argument";
        return LFD_EINVAL;
    }
    const Geo& g = ctx->g;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int64_t nvol = (int64_t)g.Nz * g.H * g.W, nimg = (int64_t)g.H * g.W;
    const bool vdev = is_device_ptr(v), ydev = is_device_ptr(y_out);
    const float* vd = v;
    if (!vdev) {
        LFD_TRY(ensure_stage(ctx, true));
        LFD_CK(cudaMemcpyAsync(ctx->stage_vol, v, nvol * sizeof(float), cudaMemcpyHostToDevice, st));
        vd = ctx->stage_vol;
    }
    float* yd = y_out;
    if (!ydev) {
        LFD_TRY(ensure_stage(ctx, false));
        yd = ctx->stage_img;
    }
    ctx->split_cur = -1;  // the iterate buffers are reused below
    if (ctx->fft) {
        const FftPlan& fp = *static_cast<const FftPlan*>(ctx->fft);
        LFD_CK(launch_poly_volume_cm(vd, g, ctx->Vcm[0], st));
        LFD_CK(fft_forward(fp, g, fbufs(ctx), 1, ctx->Vcm[0], yd, nullptr, nullptr, nullptr, 0.f, st,
                           nullptr));
    } else {
        LFD_CK(launch_poly_volume(vd, g, ctx->Vp32[0], ctx->Vpb[0], ctx->Vpb[1], st));
        LFD_TRY(run_forward(ctx, 0, st));
        LFD_CK(launch_fwd_finish_image(ctx->Fwd, fwd_parts(ctx), g, yd, st));
    }
    if (!ydev) {
        LFD_CK(cudaMemcpyAsync(y_out, yd, nimg * sizeof(float), cudaMemcpyDeviceToHost, st));
        LFD_CK(cudaStreamSynchronize(st));
    }
    return LFD_OK;
}

lfd_status lfd_backward(lfd_ctx* ctx, const float* r, float* v_out, void* cuda_stream) {
    if (!ctx) return LFD_EINVAL;
    if (!r || !v_out) {
        ctx->err = "NULL argument";
        return LFD_EINVAL;
    }
    const Geo& g = ctx->g;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int64_t nvol = (int64_t)g.Nz * g.H * g.W, nimg = (int64_t)g.H * g.W;
    const bool rdev = is_device_ptr(r), vdev = is_device_ptr(v_out);
    const float* rd = r;
    if (!rdev) {
        LFD_TRY(ensure_stage(ctx, false));
        LFD_CK(cudaMemcpyAsync(ctx->stage_img, r, nimg * sizeof(float), cudaMemcpyHostToDevice, st));
        rd = ctx->stage_img;
    }
    float* vd = v_out;
    if (!vdev) {
        LFD_TRY(ensure_stage(ctx, true));
        vd = ctx->stage_vol;
    }
    if (ctx->fft) {
        const FftPlan& fp = *static_cast<const FftPlan*>(ctx->fft);
        LFD_CK(launch_poly_image_cm(rd, g, ctx->Rcm, st));
        LFD_CK(fft_backward(fp, g, fbufs(ctx), 1, ctx->Rcm, ctx->Xcm, nullptr, st, nullptr));
        LFD_CK(exact_bwd(ctx->exact, 1, rd, ctx->Xcm, st));
        LFD_CK(launch_depoly_volume_cm(ctx->Xcm, g, vd, st));
    } else {
        LFD_CK(launch_poly_image(rd, g, ctx->Rp32, g.m_base, ctx->Rpb[0], ctx->Rpb[1], st));
        LFD_TRY(run_backward(ctx, st));
        LFD_CK(launch_sum_depoly_volume(ctx->Bwd, bwd_parts(ctx), g, vd, st));
    }
    if (!vdev) {
        LFD_CK(cudaMemcpyAsync(v_out, vd, nvol * sizeof(float), cudaMemcpyDeviceToHost, st));
        LFD_CK(cudaStreamSynchronize(st));
    }
    return LFD_OK;
}

// ------------------------------------------------------------ depth split --
// One RL iteration cut at its two exchange points, for a context made over a
// range of depths (Section 2.1, Fig. 1: the depths are divided among GPUs).
// The caller sums the partial forward projections of all depth ranges and
// takes the maximum of their partial z-projections and the sum of their flux
// between the calls.

lfd_status lfd_split_load(lfd_ctx* ctx, const float* v, void* cuda_stream) {
    if (!ctx) return LFD_EINVAL;
    if (!v) {
        ctx->err = "NULL argument";
        return LFD_EINVAL;
    }
    const Geo& g = ctx->g;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const float* vd = v;
    if (!is_device_ptr(v)) {
        LFD_TRY(ensure_stage(ctx, true));
        LFD_CK(cudaMemcpyAsync(ctx->stage_vol, v, (int64_t)g.Nz * g.H * g.W * sizeof(float),
                               cudaMemcpyHostToDevice, st));
        vd = ctx->stage_vol;
    }
    if (ctx->fft)
        LFD_CK(launch_poly_volume_cm(vd, g, ctx->Vcm[0], st));
    else
        LFD_CK(launch_poly_volume(vd, g, ctx->Vp32[0], ctx->Vpb[0], ctx->Vpb[1], st));
    ctx->split_cur = 0;
    ctx->split_prev = 0;
    return LFD_OK;
}

lfd_status lfd_split_forward(lfd_ctx* ctx, float* hv_part, void* cuda_stream) {
    if (!ctx) return LFD_EINVAL;
    if (!hv_part || !is_device_ptr(hv_part)) {
        ctx->err = "hv_part must be device memory";
        return LFD_EINVAL;
    }
    if (ctx->split_cur < 0) {
        ctx->err = "no iterate loaded (lfd_split_load)";
        return LFD_EINVAL;
    }
    const Geo& g = ctx->g;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int cur = ctx->split_cur;
    if (ctx->fft) {
        const FftPlan& fp = *static_cast<const FftPlan*>(ctx->fft);
        LFD_CK(fft_forward(fp, g, fbufs(ctx), 1, ctx->Vcm[cur], hv_part, nullptr, nullptr, nullptr, 0.f,
                           st, nullptr));
    } else {
        LFD_TRY(run_forward(ctx, cur, st));
        LFD_CK(launch_fwd_finish_image(ctx->Fwd, fwd_parts(ctx), g, hv_part, st));
    }
    return LFD_OK;
}

lfd_status lfd_split_update(lfd_ctx* ctx, const float* y, const float* hv, float* mip_part,
                            double* flux_part, void* cuda_stream) {
    if (!ctx) return LFD_EINVAL;
    if (!y || !hv || !mip_part || !flux_part || !is_device_ptr(y) || !is_device_ptr(hv) ||
        !is_device_ptr(mip_part) || !is_device_ptr(flux_part)) {
        ctx->err = "y, hv, mip_part and flux_part must be device memory";
        return LFD_EINVAL;
    }
    if (ctx->split_cur < 0) {
        ctx->err = "no iterate loaded (lfd_split_load)";
        return LFD_EINVAL;
    }
    const Geo& g = ctx->g;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int cur = ctx->split_cur, nxt = cur ^ 1;
    const int64_t nimg = (int64_t)g.H * g.W;
    if (ctx->fft) {
        const FftPlan& fp = *static_cast<const FftPlan*>(ctx->fft);
        LFD_CK(launch_ratio_image(y, hv, ctx->opt.eps, nimg, ctx->rimg, st));
        LFD_CK(launch_poly_image_cm(ctx->rimg, g, ctx->Rcm, st));
        LFD_CK(fft_backward(fp, g, fbufs(ctx), 1, ctx->Rcm, ctx->Xcm, nullptr, st, nullptr));
        LFD_CK(exact_bwd(ctx->exact, 1, ctx->rimg, ctx->Xcm, st));
        LFD_CK(launch_update_cm(ctx->Vcm[cur], ctx->Vcm[nxt], ctx->Xcm, ctx->invcm, g, 1, mip_part,
                                ctx->flux_part, st));
    } else {
        LFD_TRY(ensure_stage(ctx, false));
        LFD_CK(launch_ratio_image(y, hv, ctx->opt.eps, nimg, ctx->stage_img, st));
        __nv_bfloat16* rhi = uses_tc(ctx) ? ctx->Rpb[0] : nullptr;
        __nv_bfloat16* rlo = uses_lo(ctx) ? ctx->Rpb[1] : nullptr;
        __nv_bfloat16* vhi = uses_tc(ctx) ? ctx->Vpb[0] : nullptr;
        __nv_bfloat16* vlo = uses_lo(ctx) ? ctx->Vpb[1] : nullptr;
        LFD_CK(launch_poly_image(ctx->stage_img, g, ctx->Rp32, g.m_base, rhi, rlo, st));
        LFD_TRY(run_backward(ctx, st));
        LFD_CK(launch_update(ctx->Vp32[cur], ctx->Vp32[nxt], vhi, vlo, ctx->Bwd, bwd_parts(ctx), ctx->invHt1,
                             g, mip_part, ctx->flux_part, st));
    }
    LFD_CK(launch_sum_doubles(ctx->flux_part, ctx->nflux, flux_part, st));
    ctx->split_cur = nxt;
    ctx->split_prev = 1;
    return LFD_OK;
}

lfd_status lfd_split_store(lfd_ctx* ctx, float* v, int previous, void* cuda_stream) {
    if (!ctx) return LFD_EINVAL;
    if (!v) {
        ctx->err = "NULL argument";
        return LFD_EINVAL;
    }
    if (ctx->split_cur < 0 || (previous && !ctx->split_prev)) {
        ctx->err = previous ? "no previous iterate (no lfd_split_update since lfd_split_load)"
                            : "no iterate loaded (lfd_split_load)";
        return LFD_EINVAL;
    }
    const Geo& g = ctx->g;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int buf = previous ? ctx->split_cur ^ 1 : ctx->split_cur;
    const bool vdev = is_device_ptr(v);
    float* vd = v;
    if (!vdev) {
        LFD_TRY(ensure_stage(ctx, true));
        vd = ctx->stage_vol;
    }
    if (ctx->fft)
        LFD_CK(launch_depoly_volume_cm(ctx->Vcm[buf], g, vd, st));
    else
        LFD_CK(launch_depoly_volume(ctx->Vp32[buf], g.m_base, g, vd, st));
    if (!vdev) {
        LFD_CK(cudaMemcpyAsync(v, vd, (int64_t)g.Nz * g.H * g.W * sizeof(float), cudaMemcpyDeviceToHost, st));
        LFD_CK(cudaStreamSynchronize(st));
    }
    return LFD_OK;
}

lfd_status lfd_rl_load(lfd_ctx* ctx, const float* v, void* cuda_stream) {
    return lfd_split_load(ctx, v, cuda_stream);
}

lfd_status lfd_rl_store(lfd_ctx* ctx, float* v, void* cuda_stream) {
    return lfd_split_store(ctx, v, 0, cuda_stream);
}

lfd_status lfd_rl_step(lfd_ctx* ctx, const float* y, int n, double* entropy_hist, double* flux_hist,
                       void* cuda_stream) {
    if (!ctx) return LFD_EINVAL;
    if (!y || n < 1) {
        ctx->err = "invalid argument (NULL image or n < 1)";
        return LFD_EINVAL;
    }
    if (ctx->split_cur < 0) {
        ctx->err = "no iterate loaded (lfd_rl_load)";
        return LFD_EINVAL;
    }
    return rl_step(ctx, y, n, entropy_hist, flux_hist, (cudaStream_t)cuda_stream);
}

lfd_status lfd_quality_mip(lfd_ctx* ctx, const float* mip, double* entropy, void* cuda_stream) {
    if (!ctx) return LFD_EINVAL;
    if (!mip || !entropy) {
        ctx->err = "NULL argument";
        return LFD_EINVAL;
    }
    const Geo& g = ctx->g;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const float* md = mip;
    if (!is_device_ptr(mip)) {
        LFD_TRY(ensure_stage(ctx, false));
        LFD_CK(cudaMemcpyAsync(ctx->stage_img, mip, (int64_t)g.H * g.W * sizeof(float),
                               cudaMemcpyHostToDevice, st));
        md = ctx->stage_img;
    }
    LFD_CK(launch_metric(md, ctx->cosW, ctx->cosH, g.H, g.W, ctx->XS, ctx->YS, ctx->opt.l2_over_region,
                         ctx->G, ctx->rowE2, ctx->coef, nullptr, 0, ctx->hist, nullptr, st));
    LFD_CK(cudaMemcpyAsync(ctx->host_pinned, ctx->hist, sizeof(double), cudaMemcpyDeviceToHost, st));
    LFD_CK(cudaStreamSynchronize(st));
    *entropy = ctx->host_pinned[0];
    return LFD_OK;
}

lfd_status lfd_set_profiling(lfd_ctx* ctx, int on) {
    if (!ctx) return LFD_EINVAL;
    ctx->prof.on = on != 0;
    for (double& x : ctx->prof.sum_ms) x = 0.0;
    ctx->prof.count = 0;
    return LFD_OK;
}

lfd_status lfd_stage_times(const lfd_ctx* ctx, float* ms, int n) {
    if (!ctx || !ms || n < 0) return LFD_EINVAL;
    for (int i = 0; i < n && i < kStageSlots; ++i)
        ms[i] = ctx->prof.count ? (float)(ctx->prof.sum_ms[i] / ctx->prof.count) : 0.f;
    for (int i = kStageSlots; i < n; ++i) ms[i] = 0.f;
    return LFD_OK;
}

}  // extern "C"

namespace {

// Enqueues one RL iteration for nf frames: reads iterate buffer `cur`, writes
// the other one, leaves the frames' entropy and flux in ctx->hist. e9: ten
// events to record between stages (profiling), or null.
lfd_status iter_body(lfd_ctx* ctx, int nf, int cur, cudaStream_t st, cudaEvent_t* e9) {
    const Geo& g = ctx->g;
    const int nxt = cur ^ 1;
    auto mark = [&](int i) -> cudaError_t { return e9 ? cudaEventRecord(e9[i], st) : cudaSuccess; };
    const FftPlan* fp = static_cast<const FftPlan*>(ctx->fft);
    LFD_CK(mark(0));
    if (fp) {
        const FftBuffers fb = fbufs(ctx);
        // forward with the ratio fused into its last transform
        LFD_CK(fft_forward(*fp, g, fb, nf, ctx->Vcm[cur], nullptr, ctx->Rcm, ctx->ycm, ctx->rimg,
                           ctx->opt.eps, st, e9 ? e9 + 1 : nullptr));
        LFD_CK(mark(3));
        LFD_CK(fft_backward(*fp, g, fb, nf, ctx->Rcm, ctx->Xcm, nullptr, st, e9 ? e9 + 4 : nullptr));
        LFD_CK(mark(6));
        LFD_CK(exact_bwd(ctx->exact, nf, ctx->rimg, ctx->Xcm, st));
        LFD_CK(mark(7));
        LFD_CK(launch_update_cm(ctx->Vcm[cur], ctx->Vcm[nxt], ctx->Xcm, ctx->invcm, g, nf, ctx->mip,
                                ctx->flux_part, st));
    } else {
        const int fpart = fwd_parts(ctx), bp = bwd_parts(ctx);
        __nv_bfloat16* rhi = uses_tc(ctx) ? ctx->Rpb[0] : nullptr;
        __nv_bfloat16* rlo = uses_lo(ctx) ? ctx->Rpb[1] : nullptr;
        __nv_bfloat16* vhi = uses_tc(ctx) ? ctx->Vpb[0] : nullptr;
        __nv_bfloat16* vlo = uses_lo(ctx) ? ctx->Vpb[1] : nullptr;
        LFD_CK(mark(1));
        LFD_TRY(run_forward(ctx, cur, st));
        LFD_CK(mark(2));
        LFD_CK(launch_fwd_finish_ratio(ctx->Fwd, fpart, ctx->ypoly, ctx->opt.eps, g, ctx->Rp32, rhi, rlo, st));
        LFD_CK(mark(3));
        LFD_CK(mark(4));
        LFD_TRY(run_backward(ctx, st));
        LFD_CK(mark(5));
        LFD_CK(mark(6));
        LFD_CK(mark(7));
        LFD_CK(launch_update(ctx->Vp32[cur], ctx->Vp32[nxt], vhi, vlo, ctx->Bwd, bp, ctx->invHt1, g,
                             ctx->mip, ctx->flux_part, st));
    }
    LFD_CK(mark(8));
    LFD_CK(launch_metric(ctx->mip, ctx->cosW, ctx->cosH, g.H, g.W, ctx->XS, ctx->YS,
                         ctx->opt.l2_over_region, ctx->G, ctx->rowE2, ctx->coef, ctx->flux_part,
                         ctx->nflux, ctx->hist, ctx->hist + ctx->mf, st, nf, 1));
    LFD_CK(mark(9));
    return LFD_OK;
}

// (re)captures the two iteration graphs for nf frames
lfd_status ensure_graphs(lfd_ctx* ctx, int nf) {
    if (ctx->graph[0] && ctx->graph_nf == nf) return LFD_OK;
    for (auto& ge : ctx->graph)
        if (ge) {
            cudaGraphExecDestroy(ge);
            ge = nullptr;
        }
    for (int cur = 0; cur < 2; ++cur) {
        const uint64_t before = g_launches.load();
        LFD_CK(cudaStreamBeginCapture(ctx->wstream, cudaStreamCaptureModeRelaxed));
        lfd_status s = iter_body(ctx, nf, cur, ctx->wstream, nullptr);
        cudaGraph_t graph = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(ctx->wstream, &graph);
        g_launches.store(before);  // capture enqueues nothing; replays are counted
        if (s != LFD_OK) {
            if (graph) cudaGraphDestroy(graph);
            return s;
        }
        LFD_CK(ec);
        ctx->graph_launches = 0;
        size_t nnodes = 0;
        LFD_CK(cudaGraphGetNodes(graph, nullptr, &nnodes));
        ctx->graph_launches = nnodes;
        const cudaError_t ei = cudaGraphInstantiate(&ctx->graph[cur], graph, 0);
        cudaGraphDestroy(graph);
        LFD_CK(ei);
    }
    ctx->graph_nf = nf;
    return LFD_OK;
}

lfd_status rl_run(lfd_ctx* ctx, int nf, const float* y, float* v, int n, int stop_at_predicted,
                  int* iters_done, int* predicted, double* entropy_hist, double* flux_hist,
                  cudaStream_t ust) {
    if (!y || !v || n < 1) {
        ctx->err = "invalid argument (NULL pointer or n < 1)";
        return LFD_EINVAL;
    }
    if (nf < 1 || nf > ctx->mf) {
        ctx->err = "nframes must lie in 1 .. max_frames (" + std::to_string(ctx->mf) + ")";
        return LFD_EINVAL;
    }
    const Geo& g = ctx->g;
    const int64_t nvol = (int64_t)g.Nz * g.H * g.W, nimg = (int64_t)g.H * g.W, L2 = (int64_t)g.Ly * g.Lx;
    const bool prof = ctx->prof.on;
    ctx->split_cur = -1;  // the iterate buffers are reused below
    const bool graphs = ctx->opt.use_graph && !prof;
    // all work runs on the context's stream, ordered after the caller's
    cudaStream_t st = ctx->wstream;
    LFD_CK(cudaEventRecord(ctx->ev_in, ust));
    LFD_CK(cudaStreamWaitEvent(st, ctx->ev_in, 0));
    if ((int64_t)n * nf > (int64_t)ctx->host_hist_n * ctx->mf || !ctx->host_hist) {
        if (ctx->host_hist) cudaFreeHost(ctx->host_hist);
        ctx->host_hist = nullptr;
        LFD_CK(cudaMallocHost((void**)&ctx->host_hist, 2 * sizeof(double) * (size_t)n * ctx->mf));
        ctx->host_hist_n = n;
    }
    double* hE = ctx->host_hist;            // [nf][n]
    double* hF = ctx->host_hist + (size_t)nf * n;
    const bool ydev = is_device_ptr(y), vdev = is_device_ptr(v);
    const float* yd = y;
    float* vd = v;
    if (!ydev) {
        LFD_TRY(ensure_stage(ctx, false));
        LFD_CK(cudaMemcpyAsync(ctx->stage_img, y, nf * nimg * sizeof(float), cudaMemcpyHostToDevice, st));
        yd = ctx->stage_img;
    }
    if (!vdev) {
        LFD_TRY(ensure_stage(ctx, true));
        LFD_CK(cudaMemcpyAsync(ctx->stage_vol, v, nf * nvol * sizeof(float), cudaMemcpyHostToDevice, st));
        vd = ctx->stage_vol;
    }
    const FftPlan* fp = static_cast<const FftPlan*>(ctx->fft);
    int cur = 0;
    for (int f = 0; f < nf; ++f) {
        if (fp) {
            LFD_CK(launch_poly_image_cm(yd + f * nimg, g, ctx->ycm + f * g.S * L2, st));
            LFD_CK(launch_poly_volume_cm(vd + f * nvol, g, ctx->Vcm[cur] + f * g.C * L2, st));
        } else {
            LFD_CK(launch_poly_image(yd, g, ctx->ypoly, 0, nullptr, nullptr, st));
            LFD_CK(launch_poly_volume(vd, g, ctx->Vp32[cur], ctx->Vpb[0], ctx->Vpb[1], st));
        }
    }
    constexpr int kEv = 10;  // events per iteration (see lfd_stage_times)
    if (prof && ctx->prof.ev.size() < kEv * (size_t)n) {
        const size_t old = ctx->prof.ev.size();
        ctx->prof.ev.resize(kEv * (size_t)n, nullptr);
        for (size_t i = old; i < ctx->prof.ev.size(); ++i) LFD_CK(cudaEventCreate(&ctx->prof.ev[i]));
    }
    cudaEvent_t* ev = prof ? ctx->prof.ev.data() : nullptr;
    if (graphs) LFD_TRY(ensure_graphs(ctx, nf));

    // per frame: still iterating, iterations whose result is final, iterations run.
    // Slots 0 .. nact-1 hold the frames still iterating (slot_frame[s]); with
    // stop_at_predicted a stopped frame leaves its slot and the last active
    // slot moves into it, so later iterations only process active frames.
    std::vector<char> active(nf, 1);
    std::vector<int> done(nf, 0), ran_f(nf, 0), slot_frame(nf);
    for (int f = 0; f < nf; ++f) slot_frame[f] = f;
    int ran = 0, nact = nf;
    auto deposit = [&](int f, int slot, int buf) -> cudaError_t {  // frame f's result from a slot of buf
        if (fp) return launch_depoly_volume_cm(ctx->Vcm[buf] + slot * g.C * L2, g, vd + f * nvol, st);
        return launch_depoly_volume(ctx->Vp32[buf], g.m_base, g, vd, st);
    };
    for (int k = 0; k < n; ++k) {
        if (graphs) {
            LFD_TRY(ensure_graphs(ctx, nact));
            LFD_CK(cudaGraphLaunch(ctx->graph[cur], st));
            count_launch(ctx->graph_launches);
        } else {
            LFD_TRY(iter_body(ctx, nact, cur, st, prof ? ev + kEv * k : nullptr));
        }
        ran = k + 1;
        if (!stop_at_predicted) {
            // slots never move: this iteration's values go straight to the histories
            LFD_CK(cudaMemcpy2DAsync(hE + k, n * sizeof(double), ctx->hist, sizeof(double), sizeof(double),
                                     nf, cudaMemcpyDeviceToHost, st));
            LFD_CK(cudaMemcpy2DAsync(hF + k, n * sizeof(double), ctx->hist + ctx->mf, sizeof(double),
                                     sizeof(double), nf, cudaMemcpyDeviceToHost, st));
            for (int f = 0; f < nf; ++f) ran_f[f] = ran;
            cur ^= 1;
            continue;
        }
        LFD_CK(cudaMemcpyAsync(ctx->host_pinned_slots, ctx->hist, nact * sizeof(double),
                               cudaMemcpyDeviceToHost, st));
        LFD_CK(cudaMemcpyAsync(ctx->host_pinned_slots + ctx->mf, ctx->hist + ctx->mf, nact * sizeof(double),
                               cudaMemcpyDeviceToHost, st));
        LFD_CK(cudaStreamSynchronize(st));
        const int nxt = cur ^ 1;
        std::vector<char> freed(nact, 0);
        for (int s2 = 0; s2 < nact; ++s2) {
            const int f = slot_frame[s2];
            hE[(size_t)f * n + k] = ctx->host_pinned_slots[s2];
            hF[(size_t)f * n + k] = ctx->host_pinned_slots[ctx->mf + s2];
            ran_f[f] = ran;
            // E_{k+1} < E_k: frame f keeps v^k, still in buffer cur
            if (k >= 1 && hE[(size_t)f * n + k] < hE[(size_t)f * n + k - 1]) {
                LFD_CK(deposit(f, s2, cur));
                active[f] = 0;
                done[f] = k;
                freed[s2] = 1;
            }
        }
        // compact: the highest active slots move down into the freed ones
        int hi = nact - 1;
        for (int s2 = 0; s2 < nact; ++s2) {
            if (!freed[s2]) continue;
            while (hi > s2 && freed[hi]) --hi;
            if (hi <= s2) break;
            if (fp) {
                LFD_CK(cudaMemcpyAsync(ctx->Vcm[nxt] + s2 * g.C * L2, ctx->Vcm[nxt] + hi * g.C * L2,
                                       g.C * L2 * sizeof(float), cudaMemcpyDeviceToDevice, st));
                LFD_CK(cudaMemcpyAsync(ctx->ycm + s2 * g.S * L2, ctx->ycm + hi * g.S * L2,
                                       g.S * L2 * sizeof(float), cudaMemcpyDeviceToDevice, st));
            }
            slot_frame[s2] = slot_frame[hi];
            freed[s2] = 0;
            freed[hi] = 1;
            --hi;
        }
        int na = 0;
        for (int s2 = 0; s2 < nact; ++s2) na += freed[s2] ? 0 : 1;
        nact = na;
        cur = nxt;
        if (nact == 0) break;
    }
    for (int s2 = 0; s2 < nact; ++s2) {
        const int f = slot_frame[s2];
        if (active[f]) {
            LFD_CK(deposit(f, s2, cur));
            done[f] = ran;
        }
    }
    if (!vdev) LFD_CK(cudaMemcpyAsync(v, vd, nf * nvol * sizeof(float), cudaMemcpyDeviceToHost, st));
    LFD_CK(cudaEventRecord(ctx->ev_out, st));
    LFD_CK(cudaStreamWaitEvent(ust, ctx->ev_out, 0));
    LFD_CK(cudaStreamSynchronize(st));
    if (ctx->cg) {
        const int te = cgemm_error(ctx->cg);
        if (te != 0) {
            ctx->err = "tensor-core contraction gave up waiting (code " + std::to_string(te) + ")";
            return LFD_ETIMEDOUT;
        }
    }
    if (uses_tc(ctx)) {
        const int te = tc_error(ctx);
        if (te != 0) {
            ctx->err = "tensor-core kernel gave up waiting (code " + std::to_string(te) + ")";
            return LFD_ETIMEDOUT;
        }
    }
    if (prof) {
        for (int k = 0; k < ran; ++k) {
            float t[kEv];
            t[0] = 0.f;
            for (int i = 1; i < kEv; ++i)
                LFD_CK(cudaEventElapsedTime(&t[i], ev[kEv * k], ev[kEv * k + i]));
            const bool f = fp != nullptr;
            double* sm = ctx->prof.sum_ms;
            sm[0] += f ? t[3] : t[2];                        // forward projection
            sm[1] += f ? 0.0 : t[3] - t[2];                  // ratio (fused in the FFT variant)
            sm[2] += t[7] - t[3];                            // backprojection
            sm[3] += t[8] - t[7];                            // update
            sm[4] += t[9] - t[8];                            // metric
            sm[5] += t[2] - t[1];                            // forward contraction
            sm[6] += t[5] - t[4];                            // backward contraction
            sm[7] += f ? t[1] + (t[3] - t[2]) + (t[4] - t[3]) + (t[6] - t[5]) : 0.0;  // transforms
            sm[8] += f ? t[1] : 0.0;                         // volume R2C (forward input)
            sm[9] += f ? t[6] - t[5] : 0.0;                  // volume C2R (backward output)
            sm[10] += f ? t[7] - t[6] : 0.0;                 // exact low-sensitivity backprojection
        }
        ctx->prof.count += ran;
    }
    for (int f = 0; f < nf; ++f) {
        const double* Ef = hE + (size_t)f * n;
        const double* Ff = hF + (size_t)f * n;
        if (entropy_hist)
            for (int k = 0; k < n; ++k) entropy_hist[(size_t)f * n + k] = k < ran_f[f] ? Ef[k] : NAN;
        if (flux_hist)
            for (int k = 0; k < n; ++k) flux_hist[(size_t)f * n + k] = k < ran_f[f] ? Ff[k] : NAN;
        if (iters_done) iters_done[f] = done[f];
        if (predicted) predicted[f] = lfd_predict_stop(Ef, ran_f[f]);
    }
    return LFD_OK;
}

// n iterations of the resident iterate (buffer ctx->split_cur, frame 0) with
// the image y; leaves the result resident and the per-iteration entropy and
// flux in the host arrays (may be null)
lfd_status rl_step(lfd_ctx* ctx, const float* y, int n, double* entropy_hist, double* flux_hist,
                   cudaStream_t ust) {
    const Geo& g = ctx->g;
    const bool prof = ctx->prof.on;
    const bool graphs = ctx->opt.use_graph && !prof;
    cudaStream_t st = ctx->wstream;
    LFD_CK(cudaEventRecord(ctx->ev_in, ust));
    LFD_CK(cudaStreamWaitEvent(st, ctx->ev_in, 0));
    if ((int64_t)n > (int64_t)ctx->host_hist_n * ctx->mf || !ctx->host_hist) {
        if (ctx->host_hist) cudaFreeHost(ctx->host_hist);
        ctx->host_hist = nullptr;
        LFD_CK(cudaMallocHost((void**)&ctx->host_hist, 2 * sizeof(double) * (size_t)n * ctx->mf));
        ctx->host_hist_n = n;
    }
    double* hE = ctx->host_hist;
    double* hF = ctx->host_hist + n;
    const float* yd = y;
    if (!is_device_ptr(y)) {
        LFD_TRY(ensure_stage(ctx, false));
        LFD_CK(cudaMemcpyAsync(ctx->stage_img, y, (int64_t)g.H * g.W * sizeof(float), cudaMemcpyHostToDevice,
                               st));
        yd = ctx->stage_img;
    }
    if (ctx->fft)
        LFD_CK(launch_poly_image_cm(yd, g, ctx->ycm, st));
    else
        LFD_CK(launch_poly_image(yd, g, ctx->ypoly, 0, nullptr, nullptr, st));
    if (graphs) LFD_TRY(ensure_graphs(ctx, 1));
    int cur = ctx->split_cur;
    for (int k = 0; k < n; ++k) {
        if (graphs) {
            LFD_CK(cudaGraphLaunch(ctx->graph[cur], st));
            count_launch(ctx->graph_launches);
        } else {
            LFD_TRY(iter_body(ctx, 1, cur, st, nullptr));
        }
        LFD_CK(cudaMemcpyAsync(hE + k, ctx->hist, sizeof(double), cudaMemcpyDeviceToHost, st));
        LFD_CK(cudaMemcpyAsync(hF + k, ctx->hist + ctx->mf, sizeof(double), cudaMemcpyDeviceToHost, st));
        cur ^= 1;
    }
    ctx->split_cur = cur;
    ctx->split_prev = 1;
    LFD_CK(cudaEventRecord(ctx->ev_out, st));
    LFD_CK(cudaStreamWaitEvent(ust, ctx->ev_out, 0));
    LFD_CK(cudaStreamSynchronize(st));
    if (ctx->cg) {
        const int te = cgemm_error(ctx->cg);
        if (te != 0) {
            ctx->err = "tensor-core contraction gave up waiting (code " + std::to_string(te) + ")";
            return LFD_ETIMEDOUT;
        }
    }
    if (uses_tc(ctx)) {
        const int te = tc_error(ctx);
        if (te != 0) {
            ctx->err = "tensor-core kernel gave up waiting (code " + std::to_string(te) + ")";
            return LFD_ETIMEDOUT;
        }
    }
    for (int k = 0; k < n; ++k) {
        if (entropy_hist) entropy_hist[k] = hE[k];
        if (flux_hist) flux_hist[k] = hF[k];
    }
    return LFD_OK;
}

}  // namespace

extern "C" {

lfd_status lfd_rl_iterate(lfd_ctx* ctx, const float* y, float* v, int n, int stop_at_predicted,
                          int* iters_done, int* predicted, double* entropy_hist, double* flux_hist,
                          void* cuda_stream) {
    if (!ctx) return LFD_EINVAL;
    return rl_run(ctx, 1, y, v, n, stop_at_predicted, iters_done, predicted, entropy_hist, flux_hist,
                  (cudaStream_t)cuda_stream);
}

lfd_status lfd_rl_iterate_batch(lfd_ctx* ctx, int nframes, const float* y, float* v, int n,
                                int stop_at_predicted, int* iters_done, int* predicted,
                                double* entropy_hist, double* flux_hist, void* cuda_stream) {
    if (!ctx) return LFD_EINVAL;
    return rl_run(ctx, nframes, y, v, n, stop_at_predicted, iters_done, predicted, entropy_hist,
                  flux_hist, (cudaStream_t)cuda_stream);
}

lfd_status lfd_quality(lfd_ctx* ctx, const float* v, double* entropy, void* cuda_stream) {
    if (!ctx) return LFD_EINVAL;
    if (!v || !entropy) {
        ctx->err = "NULL argument";
        return LFD_EINVAL;
    }
    const Geo& g = ctx->g;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int64_t nvol = (int64_t)g.Nz * g.H * g.W;
    const float* vd = v;
    if (!is_device_ptr(v)) {
        LFD_TRY(ensure_stage(ctx, true));
        LFD_CK(cudaMemcpyAsync(ctx->stage_vol, v, nvol * sizeof(float), cudaMemcpyHostToDevice, st));
        vd = ctx->stage_vol;
    }
    LFD_CK(launch_mip_stack(vd, g.Nz, (int64_t)g.H * g.W, ctx->mip, st));
    LFD_CK(launch_metric(ctx->mip, ctx->cosW, ctx->cosH, g.H, g.W, ctx->XS, ctx->YS,
                         ctx->opt.l2_over_region, ctx->G, ctx->rowE2, ctx->coef, nullptr, 0,
                         ctx->hist, nullptr, st));
    LFD_CK(cudaMemcpyAsync(ctx->host_pinned, ctx->hist, sizeof(double), cudaMemcpyDeviceToHost, st));
    LFD_CK(cudaStreamSynchronize(st));
    *entropy = ctx->host_pinned[0];
    return LFD_OK;
}

}  // extern "C"

namespace {

// one batched RL iteration of opt's context, timed with CUDA events (ms), or
// a status other than LFD_OK
lfd_status time_tiles(const float* psf, int P, int Nnum, int Nz, int H, int W, const lfd_options& o,
                      cudaStream_t st, float* ms_out) {
    const int nf = o.max_frames;
    const int64_t nimg = (int64_t)nf * H * W, nvol = (int64_t)nf * Nz * H * W;
    lfd_ctx* ctx = nullptr;
    lfd_status s = lfd_create(psf, P, Nnum, Nz, H, W, &o, st, &ctx);
    if (s != LFD_OK) return s;
    float* y = nullptr;
    float* v = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    float ms = -1.f;
    bool ok = cudaMalloc(&y, nimg * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&v, nvol * sizeof(float)) == cudaSuccess &&
              cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess;
    ok = ok && launch_fill(y, nimg, 10.f, st) == cudaSuccess && launch_fill(v, nvol, 1.f, st) == cudaSuccess;
    ok = ok && lfd_rl_iterate_batch(ctx, nf, y, v, 1, 0, nullptr, nullptr, nullptr, nullptr, st) == LFD_OK;
    ok = ok && cudaEventRecord(a, st) == cudaSuccess &&
         lfd_rl_iterate_batch(ctx, nf, y, v, 2, 0, nullptr, nullptr, nullptr, nullptr, st) == LFD_OK &&
         cudaEventRecord(b, st) == cudaSuccess && cudaEventSynchronize(b) == cudaSuccess &&
         cudaEventElapsedTime(&ms, a, b) == cudaSuccess;
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (y) cudaFree(y);
    if (v) cudaFree(v);
    lfd_destroy(ctx);
    if (!ok) {
        cudaGetLastError();
        return LFD_ECUDA;
    }
    *ms_out = 0.5f * ms;
    return LFD_OK;
}

// the fastest (fft_size, contraction_cols) of the candidates
lfd_status tune_tiles(const float* psf, int P, int Nnum, int Nz, int H, int W, const lfd_options& base,
                      cudaStream_t st, bool tune_cols, int* bestF, int* bestCols, float* best_ms) {
    Geo g;
    std::string why;
    if (!make_geo(P, Nnum, Nz, H, W, &g, &why)) return LFD_EINVAL;
    const int products = base.precision == LFD_BF16X3 ? 3 : base.precision == LFD_BF16 ? 2 : 0;
    float best = 0.f;
    int bF = 0, bC = 0;
    lfd_status last = LFD_EUNSUPPORTED;
    for (int F : {32, 64}) {
        FftPlan plan{};
        if (!fft_plan_for(g, &plan, F, base.max_frames, products)) continue;
        const int need = std::min(64, (base.max_frames * plan.ntile + 15) / 16 * 16);
        std::vector<int> cols;
        if (!tune_cols || products == 0) cols.push_back(base.contraction_cols);
        else
            for (int c : {16, 32, 64})
                if (c <= need) cols.push_back(c);
        for (int c : cols) {
            lfd_options o = base;
            o.fft_size = F;
            o.contraction_cols = c;
            o.use_graph = 1;
            float ms = 0.f;
            const lfd_status s = time_tiles(psf, P, Nnum, Nz, H, W, o, st, &ms);
            if (s != LFD_OK) {
                if (s != LFD_EUNSUPPORTED) last = s;
                continue;
            }
            if (bF == 0 || ms < best) {
                best = ms;
                bF = F;
                bC = c;
            }
        }
    }
    if (bF == 0) return last;
    *bestF = bF;
    *bestCols = bC;
    *best_ms = best;
    return LFD_OK;
}

struct TuneResult {
    int F, cols;
    float ms;
};
std::mutex g_tune_mu;
std::map<std::string, TuneResult> g_tune_cache;

// cache key: the PSF (address and 16 of its values spread over the array),
// the shape, the frames and the options that change the tiles' cost
bool tune_key(const float* psf, int P, int Nnum, int Nz, int H, int W, const lfd_options& o, std::string* key) {
    const int64_t count = (int64_t)Nz * Nnum * Nnum * P * P;
    uint32_t sample[16];
    for (int k = 0; k < 16; ++k) {
        float x = 0.f;
        if (cudaMemcpy(&x, psf + count * k / 16, sizeof(float), cudaMemcpyDefault) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        std::memcpy(&sample[k], &x, sizeof(x));
    }
    int dev = 0;
    cudaGetDevice(&dev);
    char buf[256];
    std::snprintf(buf, sizeof(buf), "%d|%p|%d|%d|%d|%d|%d|%d|%d|%a|", dev, (const void*)psf, P, Nnum, Nz, H, W,
                  o.max_frames, o.precision, (double)o.spectra_lo_tau);
    *key = buf;
    for (uint32_t v : sample) *key += std::to_string(v) + ",";
    return true;
}

}  // namespace

extern "C" {

lfd_status lfd_autotune(const float* psf, int P, int Nnum, int Nz, int H, int W,
                        const lfd_options* opt, void* cuda_stream, int* best_size,
                        float* ms_per_iter) {
    if (!psf || !opt || !best_size || opt->variant != LFD_FFT) return LFD_EINVAL;
    int F = 0, cols = 0;
    float ms = 0.f;
    const lfd_status s = tune_tiles(psf, P, Nnum, Nz, H, W, *opt, (cudaStream_t)cuda_stream, false, &F, &cols, &ms);
    if (s != LFD_OK) return s;
    *best_size = F;
    if (ms_per_iter) *ms_per_iter = ms;
    return LFD_OK;
}

lfd_status lfd_autotune_options(const float* psf, int P, int Nnum, int Nz, int H, int W,
                                lfd_options* opt, void* cuda_stream, float* ms_per_iter, int* cached) {
    if (!psf || !opt || opt->variant != LFD_FFT || opt->max_frames < 1) return LFD_EINVAL;
    if (cached) *cached = 0;
    std::string key;
    const bool keyed = tune_key(psf, P, Nnum, Nz, H, W, *opt, &key);
    if (keyed) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            opt->fft_size = it->second.F;
            opt->contraction_cols = it->second.cols;
            if (ms_per_iter) *ms_per_iter = it->second.ms;
            if (cached) *cached = 1;
            return LFD_OK;
        }
    }
    int F = 0, cols = 0;
    float ms = 0.f;
    const lfd_status s = tune_tiles(psf, P, Nnum, Nz, H, W, *opt, (cudaStream_t)cuda_stream, true, &F, &cols, &ms);
    if (s != LFD_OK) return s;
    opt->fft_size = F;
    opt->contraction_cols = cols;
    if (ms_per_iter) *ms_per_iter = ms;
    if (keyed) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = TuneResult{F, cols, ms};
    }
    return LFD_OK;
}

}  // extern "C"
