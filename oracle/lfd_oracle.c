/*
 * Light-field projection oracle: plain, slow, FP64 direct summation.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product library links, includes or
 * calls this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark load it. It shares no code, header or table with the CUDA path.
 *
 * Model (the light-field forward model that the paper deconvolves with
 * Richardson-Lucy, Section 1 and Section 2.1; the paper does not write it out,
 * so it is restated here in the form of Prevedel et al. 2014 that the paper
 * builds on):
 *
 *   volume v[z][i'][j'], z < Nz, i' < H, j' < W       (lateral grid = sensor grid)
 *   PSF    K[z][aa][bb][mi][mj], aa,bb < Nnum, mi,mj < P, P odd, centre c=(P-1)/2
 *   phase of a voxel (i',j') = (i' mod Nnum, j' mod Nnum)
 *
 *   forward   (Hv)[i][j]        = sum_z sum_{i',j'} v[z][i'][j'] *
 *                                   K[z][i'%N][j'%N][i-i'+c][j-j'+c]
 *   backward  (H^T r)[z][i'][j'] = sum_{i,j} r[i][j] *
 *                                   K[z][i'%N][j'%N][i-i'+c][j-j'+c]
 *
 * with every term whose PSF index falls outside [0,P) or whose pixel falls
 * outside the sensor dropped (zero padding). The backward sum is exactly the
 * transpose of the forward sum: the same coefficient links voxel (z,i',j') and
 * pixel (i,j) in both.
 *
 * Arithmetic: inputs are converted to double by the caller; every product and
 * sum is FP64. Compile with -ffp-contract=off so x86 and Arm give the same bits.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define PSF_AT(psf, N, P, z, aa, bb) \
    ((psf) + ((((size_t)(z) * (N) + (aa)) * (N) + (bb)) * (size_t)(P) * (P)))

static int imax(int a, int b) { return a > b ? a : b; }
static int imin(int a, int b) { return a < b ? a : b; }

typedef struct {
    const double *psf;
    int P, N, Nz, H, W;
    const double *in;
    double *out;
    const int *idx;  /* sampled variants: coordinates */
    long lo, hi;     /* this thread's share */
} job_t;

/* run fn over [0,total) split in nthreads contiguous shares */
static void run_jobs(void *(*fn)(void *), job_t base, long total, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if ((long)nthreads > total) nthreads = (int)(total > 0 ? total : 1);
    pthread_t th[256];
    job_t jobs[256];
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = base;
        jobs[t].lo = total * t / nthreads;
        jobs[t].hi = total * (t + 1) / nthreads;
    }
    for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, fn, &jobs[t]);
    fn(&jobs[0]);
    for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
}

/* ---------------------------------------------------------------- forward --
 * Each thread owns a band of output rows [lo,hi) and adds, for every voxel,
 * that voxel's PSF (the one of its own phase and depth) centred on the voxel,
 * restricted to the band. Voxels equal to zero add exact zeros and are skipped;
 * the sum is unchanged by the skip.                                           */
static void *fwd_band(void *arg) {
    const job_t *j = (const job_t *)arg;
    const int P = j->P, N = j->N, H = j->H, W = j->W, c = (P - 1) / 2;
    const int r0 = (int)j->lo, r1 = (int)j->hi;
    for (long p = (long)r0 * W; p < (long)r1 * W; ++p) j->out[p] = 0.0;
    for (int z = 0; z < j->Nz; ++z) {
        for (int ip = imax(0, r0 - c); ip < imin(H, r1 + c); ++ip) {
            const int aa = ip % N;
            const double *vrow = j->in + ((size_t)z * H + ip) * W;
            const int mi_lo = imax(0, r0 - ip + c), mi_hi = imin(P, r1 - ip + c);
            for (int jp = 0; jp < W; ++jp) {
                const double v = vrow[jp];
                if (v == 0.0) continue;
                const double *K = PSF_AT(j->psf, N, P, z, aa, jp % N);
                const int mj_lo = imax(0, c - jp), mj_hi = imin(P, W + c - jp);
                for (int mi = mi_lo; mi < mi_hi; ++mi) {
                    double *o = j->out + (size_t)(ip + mi - c) * W + (jp - c);
                    const double *k = K + (size_t)mi * P;
                    for (int mj = mj_lo; mj < mj_hi; ++mj) o[mj] += v * k[mj];
                }
            }
        }
    }
    return NULL;
}

void orc_forward(const double *psf, int P, int N, int Nz, int H, int W,
                 const double *v, double *out, int nthreads) {
    job_t b = {psf, P, N, Nz, H, W, v, out, NULL, 0, 0};
    run_jobs(fwd_band, b, H, nthreads);
}

/* --------------------------------------------------------------- backward --
 * Each voxel gathers the sensor pixels its PSF touches, weighted by that PSF.
 * Four neighbouring voxels of one row are summed side by side (independent
 * accumulators); each sum still runs over the taps in row-major order.        */
static double bwd_one(const job_t *j, int z, int ip, int jp) {
    const int P = j->P, N = j->N, H = j->H, W = j->W, c = (P - 1) / 2;
    const double *K = PSF_AT(j->psf, N, P, z, ip % N, jp % N);
    const int mi_lo = imax(0, c - ip), mi_hi = imin(P, H + c - ip);
    const int mj_lo = imax(0, c - jp), mj_hi = imin(P, W + c - jp);
    double s = 0.0;
    for (int mi = mi_lo; mi < mi_hi; ++mi) {
        const double *r = j->in + (size_t)(ip + mi - c) * W + (jp - c);
        const double *k = K + (size_t)mi * P;
        for (int mj = mj_lo; mj < mj_hi; ++mj) s += r[mj] * k[mj];
    }
    return s;
}

static void *bwd_rows(void *arg) {
    const job_t *j = (const job_t *)arg;
    const int P = j->P, N = j->N, H = j->H, W = j->W, c = (P - 1) / 2;
    for (long zr = j->lo; zr < j->hi; ++zr) {
        const int z = (int)(zr / H), ip = (int)(zr % H);
        double *orow = j->out + ((size_t)z * H + ip) * W;
        const int mi_lo = imax(0, c - ip), mi_hi = imin(P, H + c - ip);
        int jp = 0;
        /* interior block of four voxels whose windows are not clipped in x */
        for (; jp + 3 < W; jp += 4) {
            if (jp - c < 0 || jp + 3 + c >= W) {
                for (int q = 0; q < 4; ++q) orow[jp + q] = bwd_one(j, z, ip, jp + q);
                continue;
            }
            const double *K0 = PSF_AT(j->psf, N, P, z, ip % N, (jp + 0) % N);
            const double *K1 = PSF_AT(j->psf, N, P, z, ip % N, (jp + 1) % N);
            const double *K2 = PSF_AT(j->psf, N, P, z, ip % N, (jp + 2) % N);
            const double *K3 = PSF_AT(j->psf, N, P, z, ip % N, (jp + 3) % N);
            double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
            for (int mi = mi_lo; mi < mi_hi; ++mi) {
                const double *r = j->in + (size_t)(ip + mi - c) * W + (jp - c);
                const size_t o = (size_t)mi * P;
                for (int mj = 0; mj < P; ++mj) {
                    s0 += r[mj + 0] * K0[o + mj];
                    s1 += r[mj + 1] * K1[o + mj];
                    s2 += r[mj + 2] * K2[o + mj];
                    s3 += r[mj + 3] * K3[o + mj];
                }
            }
            orow[jp + 0] = s0; orow[jp + 1] = s1; orow[jp + 2] = s2; orow[jp + 3] = s3;
        }
        for (; jp < W; ++jp) orow[jp] = bwd_one(j, z, ip, jp);
    }
    return NULL;
}

void orc_backward(const double *psf, int P, int N, int Nz, int H, int W,
                  const double *r, double *out, int nthreads) {
    job_t b = {psf, P, N, Nz, H, W, r, out, NULL, 0, 0};
    run_jobs(bwd_rows, b, (long)Nz * H, nthreads);
}

/* ------------------------------------------------------- sampled outputs --
 * forward at chosen pixels idx[2q]=(i), idx[2q+1]=(j): gather form of the same
 * sum, over the voxels whose PSF reaches (i,j).                               */
static void *fwd_at(void *arg) {
    const job_t *j = (const job_t *)arg;
    const int P = j->P, N = j->N, H = j->H, W = j->W, c = (P - 1) / 2;
    for (long q = j->lo; q < j->hi; ++q) {
        const int i = j->idx[2 * q], jj = j->idx[2 * q + 1];
        double s = 0.0;
        for (int z = 0; z < j->Nz; ++z)
            for (int ip = imax(0, i - c); ip <= imin(H - 1, i + c); ++ip)
                for (int jp = imax(0, jj - c); jp <= imin(W - 1, jj + c); ++jp) {
                    const double *K = PSF_AT(j->psf, N, P, z, ip % N, jp % N);
                    s += j->in[((size_t)z * H + ip) * W + jp] *
                         K[(size_t)(i - ip + c) * P + (jj - jp + c)];
                }
        j->out[q] = s;
    }
    return NULL;
}

void orc_forward_at(const double *psf, int P, int N, int Nz, int H, int W,
                    const double *v, long npts, const int *pix, double *out,
                    int nthreads) {
    job_t b = {psf, P, N, Nz, H, W, v, out, pix, 0, 0};
    run_jobs(fwd_at, b, npts, nthreads);
}

/* backward at chosen voxels idx[3q..3q+2] = (z, i', j') */
static void *bwd_at(void *arg) {
    const job_t *j = (const job_t *)arg;
    for (long q = j->lo; q < j->hi; ++q)
        j->out[q] = bwd_one(j, j->idx[3 * q], j->idx[3 * q + 1], j->idx[3 * q + 2]);
    return NULL;
}

void orc_backward_at(const double *psf, int P, int N, int Nz, int H, int W,
                     const double *r, long npts, const int *vox, double *out,
                     int nthreads) {
    job_t b = {psf, P, N, Nz, H, W, r, out, vox, 0, 0};
    run_jobs(bwd_at, b, npts, nthreads);
}

/* number of multiply-adds one full projection performs (zero padding
 * excluded): Nz * S(H) * S(W), S(n) = sum over positions of the in-range taps */
double orc_macs(int P, int Nz, int H, int W) {
    const int c = (P - 1) / 2;
    double sh = 0.0, sw = 0.0;
    for (int i = 0; i < H; ++i) sh += imin(P, H + c - i) - imax(0, c - i);
    for (int i = 0; i < W; ++i) sw += imin(P, W + c - i) - imax(0, c - i);
    return (double)Nz * sh * sw;
}

/* ---------------------------------------------------------- voxel blocks --
 * backward at every voxel of the block [z0,z1) x [i0,i1) x [j0,j1), written
 * to out[z-z0][i'-i0][j'-j0]. Each voxel's value is the sum bwd_one forms, in
 * the same order (PSF taps row by row); eight neighbouring voxels of a row
 * whose windows lie inside the sensor along x are carried side by side, which
 * only interleaves independent sums, so the results equal backward_at's bit
 * for bit.                                                                   */
typedef struct {
    job_t j;
    int z0, i0, i1, j0, j1;
} blk_t;

static void *bwd_blk(void *arg) {
    const blk_t *b = (const blk_t *)arg;
    const job_t *j = &b->j;
    const int P = j->P, N = j->N, H = j->H, W = j->W, c = (P - 1) / 2;
    const int ni = b->i1 - b->i0, nj = b->j1 - b->j0;
    for (long zr = j->lo; zr < j->hi; ++zr) {
        const int z = b->z0 + (int)(zr / ni), ip = b->i0 + (int)(zr % ni);
        double *orow = j->out + (size_t)zr * nj;
        const int mi_lo = imax(0, c - ip), mi_hi = imin(P, H + c - ip);
        int jp = b->j0;
        for (; jp + 7 < b->j1; jp += 8) {
            if (jp - c < 0 || jp + 7 + c >= W) {
                for (int q = 0; q < 8; ++q) orow[jp + q - b->j0] = bwd_one(j, z, ip, jp + q);
                continue;
            }
            const double *K[8];
            for (int q = 0; q < 8; ++q) K[q] = PSF_AT(j->psf, N, P, z, ip % N, (jp + q) % N);
            double s[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
            for (int mi = mi_lo; mi < mi_hi; ++mi) {
                const double *r = j->in + (size_t)(ip + mi - c) * W + (jp - c);
                const size_t o = (size_t)mi * P;
                for (int mj = 0; mj < P; ++mj)
                    for (int q = 0; q < 8; ++q) s[q] += r[mj + q] * K[q][o + mj];
            }
            for (int q = 0; q < 8; ++q) orow[jp + q - b->j0] = s[q];
        }
        for (; jp < b->j1; ++jp) orow[jp - b->j0] = bwd_one(j, z, ip, jp);
    }
    return NULL;
}

void orc_backward_block(const double *psf, int P, int N, int Nz, int H, int W,
                        const double *r, int z0, int z1, int i0, int i1, int j0, int j1,
                        double *out, int nthreads) {
    const long total = (long)(z1 - z0) * (i1 - i0);
    if (total <= 0 || j1 <= j0) return;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if ((long)nthreads > total) nthreads = (int)total;
    pthread_t th[256];
    blk_t jobs[256];
    for (int t = 0; t < nthreads; ++t) {
        job_t base = {psf, P, N, Nz, H, W, r, out, NULL, total * t / nthreads,
                      total * (t + 1) / nthreads};
        blk_t b = {base, z0, i0, i1, j0, j1};
        jobs[t] = b;
    }
    for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, bwd_blk, &jobs[t]);
    bwd_blk(&jobs[0]);
    for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
}
