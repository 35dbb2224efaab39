// kf_bin.cuh -- the eta x phi bin of a point, shared by the binning kernel
// and the build's window look-up.
#pragma once

#include <cuda_runtime.h>

#include "../../include/kf.h"

namespace kfi {

constexpr float kPi = 3.14159265358979323846f;

// phi bin of an angle in [-pi, pi], clamped to [0, KF_BIN_PHI - 1]
__device__ __forceinline__ int phi_bin(float phi) {
  int b = __float2int_rd((phi + kPi) * (float(KF_BIN_PHI) / (2.0f * kPi)));
  return b < 0 ? 0 : (b >= KF_BIN_PHI ? KF_BIN_PHI - 1 : b);
}

// eta bin of eta, clamped to [0, KF_BIN_ETA - 1]
__device__ __forceinline__ int eta_bin(float eta) {
  int b = __float2int_rd((eta + KF_BIN_ETA_MAX) * (float(KF_BIN_ETA) / (2.0f * KF_BIN_ETA_MAX)));
  return b < 0 ? 0 : (b >= KF_BIN_ETA ? KF_BIN_ETA - 1 : b);
}

// Bin of a point: eta = asinh(z / r), phi = atan2(y, x).
__device__ __forceinline__ int bin_of(float x, float y, float z) {
  const float r = sqrtf(x * x + y * y);
  const float eta = r > 0.f ? asinhf(z / r) : (z >= 0.f ? 1e30f : -1e30f);
  return eta_bin(eta) * KF_BIN_PHI + phi_bin(atan2f(y, x));
}

struct BinArgs {
  const float* xyz;        // [3][stride]
  int64_t stride;
  const int64_t* seg_off;  // [n_seg + 1]
  int32_t* bin_off;        // [n_seg][KF_NBINS + 1] required: bin starts within the segment, then the count
  float4* out_pts;         // [total] or null
  int32_t* out_id;         // [total] required: id within the segment, bin order (unordered, with
                           // out_pts: scratch, left holding each point's bin in input order)
  int32_t* out_seg;        // [total] or null
  int32_t* cursor;         // [n_seg][KF_NBINS] scratch
  int unordered = 0;       // 1: leave each bin in scatter order (no sort by id)
};

// One segment of a table-driven unordered binning: points [p0, p1) of xyz
// ([3][stride]), their offsets into bin_off ([KF_NBINS + 1]), points into
// out_pts[p0 .. p1), out_id[p0 .. p1) scratch.
struct BinSegment {
  const float* xyz;
  int64_t stride;
  int64_t p0, p1;
  int32_t* bin_off;
  float4* out_pts;
  int32_t* out_id;
};
// Bin the n segments of a device table in one launch (unordered).
cudaError_t launch_bin_segment_table(const BinSegment* table, int n, cudaStream_t st);

// Sort the points of every segment into bins (several launches on `st`);
// stride is the number of points (the segments cover [seg_off[0],
// seg_off[n_segments])).
cudaError_t launch_bin_points(const BinArgs& a, int n_segments, cudaStream_t st);

}  // namespace kfi
