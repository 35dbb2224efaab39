// kf_bin.cuh -- the eta x phi bin of a point, shared by the binning kernel
// and the build's window look-up.
#pragma once

#include <cuda_runtime.h>

#include "../../include/kf.h"

namespace kfi {

constexpr float kPi = 3.14159265358979323846f;

// phi bin of an angle in [-pi, pi] among NPHI bins over [-pi, pi), clamped to
// [0, NPHI - 1].  The scale of KF_BIN_PHI_FINE sub-bins is exactly twice that
// of KF_BIN_PHI bins (a power of two), so the products differ by exactly a
// factor 2 and a sub-bin halved is the bin: floor(2a) >> 1 = floor(a).
template <int NPHI>
__device__ __forceinline__ int phi_bin_n(float phi) {
  int b = __float2int_rd((phi + kPi) * (float(NPHI) / (2.0f * kPi)));
  return b < 0 ? 0 : (b >= NPHI ? NPHI - 1 : b);
}
__device__ __forceinline__ int phi_bin(float phi) { return phi_bin_n<KF_BIN_PHI>(phi); }

// eta bin of eta, clamped to [0, KF_BIN_ETA - 1]
__device__ __forceinline__ int eta_bin(float eta) {
  int b = __float2int_rd((eta + KF_BIN_ETA_MAX) * (float(KF_BIN_ETA) / (2.0f * KF_BIN_ETA_MAX)));
  return b < 0 ? 0 : (b >= KF_BIN_ETA ? KF_BIN_ETA - 1 : b);
}

// Bin of a point: eta = asinh(z / r), phi = atan2(y, x); NPHI bins a row
// (KF_BIN_PHI: the bins, KF_BIN_PHI_FINE: the sub-bins).
template <int NPHI = KF_BIN_PHI>
__device__ __forceinline__ int bin_of(float x, float y, float z) {
  const float r = sqrtf(x * x + y * y);
  const float eta = r > 0.f ? asinhf(z / r) : (z >= 0.f ? 1e30f : -1e30f);
  return eta_bin(eta) * NPHI + phi_bin_n<NPHI>(atan2f(y, x));
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
  int32_t* fine_off = nullptr;  // unordered only: [n_seg][KF_NBINS_FINE + 1] sub-bin starts, or null;
                                // when set the points are ordered by sub-bin
};

// One segment of a table-driven unordered binning: points [p0, p1) of xyz
// ([3][stride]), their offsets into bin_off ([KF_NBINS + 1]) and, with the
// sub-bins, fine_off ([KF_NBINS_FINE + 1]), points into out_pts[p0 .. p1),
// out_id[p0 .. p1) scratch.
struct BinSegment {
  const float* xyz;
  int64_t stride;
  int64_t p0, p1;
  int32_t* bin_off;
  int32_t* fine_off;
  float4* out_pts;
  int32_t* out_id;
};
// Bin the n segments of a device table in one launch (unordered; fine: by
// sub-bin, every entry's fine_off set).
cudaError_t launch_bin_segment_table(const BinSegment* table, int n, bool fine, cudaStream_t st);

// Sort the points of every segment into bins (several launches on `st`);
// stride is the number of points (the segments cover [seg_off[0],
// seg_off[n_segments])).
cudaError_t launch_bin_points(const BinArgs& a, int n_segments, cudaStream_t st);

}  // namespace kfi
