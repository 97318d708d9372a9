// Exact backprojection of the FFT variant's low-sensitivity voxels (exact.cu).
#pragma once
#include <string>

#include "lfd_internal.h"

namespace lfd {

struct ExactPlan;

// Plans the window sums for the sorted channel-major voxel indices low[0..n)
// ([C][Ly][Lx]) of geometry g, for up to max_frames frames per call. psf is
// the device PSF [Nz][N][N][P][P]; it must outlive the plan. Device memory
// the plan allocates is added to *bytes. On failure *why says what failed.
cudaError_t exact_plan_create(const int64_t* low, int64_t n, const Geo& g, const float* psf, int max_frames,
                              cudaStream_t st, ExactPlan** out, int64_t* bytes, std::string* why);

// xcm[f][idx] = (H^T r_f)[idx] for every planned voxel idx and frame f < nf,
// by direct summation over its PSF window; rimg is [nf][H][W] (device). The
// other entries of xcm are left as they are.
cudaError_t exact_bwd(ExactPlan* p, int nf, const float* rimg, float* xcm, cudaStream_t st);

// voxels summed by runs / one warp each (for inspection and tests)
void exact_plan_counts(const ExactPlan* p, int64_t* in_runs, int64_t* runs, int64_t* single);

void exact_plan_destroy(ExactPlan* p);

}  // namespace lfd
