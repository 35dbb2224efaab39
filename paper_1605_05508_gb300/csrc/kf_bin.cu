// kf_bin.cu -- spatial partitioning of hits (and seeds) into directionally
// projective eta x phi bins per layer (Cerati et al., Sec. 3: hits sorted in
// phi within eta bins, phi bins for fast look-up of compatible hits).
//
// A counting sort with one thread block per segment (one event on one
// layer): a shared-memory histogram of the 64 x 256 bins, a block-wide
// exclusive scan, a scatter through shared-memory cursors, and a final
// insertion sort by id inside each bin so that the output is deterministic.
#include "kf_bin.cuh"
#include "kf_internal.h"

namespace kfi {

constexpr int kBinThreads = 1024;
constexpr int kPerThread = KF_NBINS / kBinThreads;  // 16 consecutive bins per thread
static_assert(KF_NBINS % kBinThreads == 0, "bins per thread");

__global__ void __launch_bounds__(kBinThreads) bin_points_kernel(const BinArgs A) {
  extern __shared__ int smem[];
  int* cnt = smem;               // [KF_NBINS] counts, then cursors
  int* warp_tot = smem + KF_NBINS;  // [32]
  const int seg = blockIdx.x;
  // offsets are clamped to the point arrays, so malformed ones cannot index past them
  int64_t p0 = A.seg_off[seg], p1 = A.seg_off[seg + 1];
  p0 = p0 < 0 ? 0 : (p0 > A.stride ? A.stride : p0);
  p1 = p1 < p0 ? p0 : (p1 > A.stride ? A.stride : p1);
  const int n = int(p1 - p0);
  const int tid = threadIdx.x;
  for (int b = tid; b < KF_NBINS; b += kBinThreads) cnt[b] = 0;
  __syncthreads();
  for (int i = tid; i < n; i += kBinThreads) {
    const int64_t g = p0 + i;
    const int b = bin_of(A.xyz[g], A.xyz[A.stride + g], A.xyz[2 * A.stride + g]);
    atomicAdd(&cnt[b], 1);
  }
  __syncthreads();
  // exclusive scan: each thread owns kPerThread consecutive bins
  int local[kPerThread];
  int run = 0;
#pragma unroll
  for (int t = 0; t < kPerThread; ++t) {
    local[t] = run;
    run += cnt[tid * kPerThread + t];
  }
  const int lane = tid & 31, warp = tid >> 5;
  int incl = run;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += v;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int w = warp_tot[lane];
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, w, d);
      if (lane >= d) w += v;
    }
    warp_tot[lane] = w;  // inclusive over warps
  }
  __syncthreads();
  const int base = (incl - run) + (warp > 0 ? warp_tot[warp - 1] : 0);
  int32_t* off = A.bin_off ? A.bin_off + int64_t(seg) * (KF_NBINS + 1) : nullptr;
#pragma unroll
  for (int t = 0; t < kPerThread; ++t) {
    const int b = tid * kPerThread + t;
    cnt[b] = base + local[t];
    if (off) off[b] = base + local[t];
  }
  if (off && tid == 0) off[KF_NBINS] = n;
  __syncthreads();
  // scatter through the cursors (order inside a bin fixed below)
  for (int i = tid; i < n; i += kBinThreads) {
    const int64_t g = p0 + i;
    const float x = A.xyz[g], y = A.xyz[A.stride + g], z = A.xyz[2 * A.stride + g];
    const int b = bin_of(x, y, z);
    const int pos = atomicAdd(&cnt[b], 1);
    A.out_id[p0 + pos] = i;
    if (A.out_pts) A.out_pts[p0 + pos] = make_float4(x, y, z, __int_as_float(i));
    if (A.out_seg) A.out_seg[p0 + pos] = seg;
  }
  __syncthreads();
  // deterministic order: insertion sort by id inside each bin (cnt[b] is now
  // the end of bin b, its start is the end of bin b - 1)
  for (int b = tid; b < KF_NBINS; b += kBinThreads) {
    const int beg = b == 0 ? 0 : cnt[b - 1], end = cnt[b];
    for (int u = beg + 1; u < end; ++u) {
      const int id = A.out_id[p0 + u];
      const float4 pt = A.out_pts ? A.out_pts[p0 + u] : make_float4(0.f, 0.f, 0.f, 0.f);
      int v = u - 1;
      while (v >= beg && A.out_id[p0 + v] > id) {
        A.out_id[p0 + v + 1] = A.out_id[p0 + v];
        if (A.out_pts) A.out_pts[p0 + v + 1] = A.out_pts[p0 + v];
        --v;
      }
      A.out_id[p0 + v + 1] = id;
      if (A.out_pts) A.out_pts[p0 + v + 1] = pt;
    }
  }
}

cudaError_t launch_bin_points(const BinArgs& a, int n_segments, cudaStream_t st) {
  if (n_segments <= 0) return cudaSuccess;
  const int smem = (KF_NBINS + 32) * int(sizeof(int));
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(bin_points_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  bin_points_kernel<<<n_segments, kBinThreads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace kfi

using namespace kfi;

extern "C" int kf_bin_hits(kf_ctx* ctx, const kf_layer_hits* in, kf_layer_hit_bins* out, void* stream) {
  if (!ctx || !in || !out) return KF_EINVAL;
  if (in->n_events < 0 || in->n_layers < 1 || in->first_layer < 0 ||
      in->first_layer + in->n_layers > ctx->cfg.n_layers || in->n_hits < 0)
    return KF_EINVAL;
  if (!in->seg_off || !out->bin_off || (in->n_hits > 0 && (!in->xyz || !out->hits))) return KF_EINVAL;
  out->n_events = in->n_events;
  out->n_layers = in->n_layers;
  out->first_layer = in->first_layer;
  out->n_hits = in->n_hits;
  out->seg_off = in->seg_off;
  const int nseg = in->n_events * in->n_layers;
  if (nseg == 0) return KF_OK;
  KF_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  int rc = scratch_reserve(ctx, ctx->s_bin_id, size_t(in->n_hits > 0 ? in->n_hits : 1) * sizeof(int32_t));
  if (rc) return rc;
  BinArgs a;
  a.xyz = in->xyz;
  a.stride = in->n_hits;
  a.seg_off = in->seg_off;
  a.bin_off = out->bin_off;
  a.out_pts = reinterpret_cast<float4*>(out->hits);
  a.out_id = static_cast<int32_t*>(ctx->s_bin_id.ptr);
  a.out_seg = nullptr;
  KF_CUDA_TRY(ctx, launch_bin_points(a, nseg, static_cast<cudaStream_t>(stream)));
  return KF_OK;
}
