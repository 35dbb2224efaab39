// kf_bin.cu -- spatial partitioning of hits (and seeds) into directionally
// projective eta x phi bins per layer (Cerati et al., Sec. 3: hits sorted in
// phi within eta bins, phi bins for fast look-up of compatible hits).
//
// A counting sort of every segment (one event on one layer) into the 64 x 256
// bins, with a final insertion sort by id inside each bin so that the output
// is deterministic (skipped with kf_tuning.bin_unordered: the build's results
// do not depend on the order of the hits inside a bin).  The unordered form
// can sort by 64 x 512 sub-bins instead, each bin two of them, and give the
// sub-bin starts as well: the build's windows then cover half as wide a
// strip of phi beyond their edges.
#include "kf_bin.cuh"
#include "kf_internal.h"

#include <algorithm>
#include <atomic>

namespace kfi {

// The ordered binning: a counting sort over all points of all segments at
// once, in four fully parallel passes: (1) every point adds one to its segment's count of its
// bin (global atomics into bin_off), (2) one block per segment turns the
// counts into exclusive offsets (bin_off) and scatter cursors, (3) every
// point takes the next slot of its bin, (4) one thread per (segment, bin)
// sorts the bin's slots by id, so the output does not depend on the order
// in which (3) took them.  A segment of any size spreads over the whole GPU.
constexpr int kScanThreads = 1024;
static_assert(KF_NBINS % kScanThreads == 0, "bins per thread");  // 16 consecutive bins a thread
constexpr int kPointThreads = 256;

// the segment s with seg_off[s] <= g < seg_off[s + 1], or -1
__device__ __forceinline__ int segment_of(const int64_t* off, int nseg, int64_t g) {
  if (g < off[0] || g >= off[nseg]) return -1;
  int lo = 0, hi = nseg - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= g)
      lo = mid;
    else
      hi = mid - 1;
  }
  return g < off[lo + 1] ? lo : -1;
}

__global__ void __launch_bounds__(kPointThreads) bin_count_kernel(const BinArgs A, int nseg) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; g < A.stride; g += stride) {
    const int s = segment_of(A.seg_off, nseg, g);
    if (s < 0) continue;
    const int b = bin_of(A.xyz[g], A.xyz[A.stride + g], A.xyz[2 * A.stride + g]);
    atomicAdd(&A.bin_off[int64_t(s) * (KF_NBINS + 1) + b], 1);
  }
}

// padded shared-memory index of bin b: a thread's 16 (or 32) consecutive
// bins and a warp's 32 threads fall in distinct banks
__device__ __forceinline__ int pad_idx(int b) { return b + (b >> 5); }
constexpr int kScanSmem = (KF_NBINS + KF_NBINS / 32) * int(sizeof(int));
// the sub-bin histogram: one block per SM
constexpr int kFineSmem = (KF_NBINS_FINE + KF_NBINS_FINE / 32) * int(sizeof(int));
static_assert(KF_NBINS_FINE % kScanThreads == 0, "sub-bins per thread");

// Exclusive scan, in place, of the NB counts in cnt (padded layout) by the
// block's kScanThreads threads, each owning NB / kScanThreads consecutive
// bins; returns the total to every thread.  Ends with a barrier.
template <int NB = KF_NBINS>
__device__ __forceinline__ int scan_bins(int* cnt, int* warp_tot) {
  constexpr int kPer = NB / kScanThreads;
  const int tid = threadIdx.x;
  int run = 0;
#pragma unroll
  for (int t = 0; t < kPer; ++t) run += cnt[pad_idx(tid * kPer + t)];
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
  int acc = (incl - run) + (warp > 0 ? warp_tot[warp - 1] : 0);
  const int total = warp_tot[kScanThreads / 32 - 1];
#pragma unroll
  for (int t = 0; t < kPer; ++t) {
    const int i = pad_idx(tid * kPer + t);
    const int c = cnt[i];
    cnt[i] = acc;
    acc += c;
  }
  __syncthreads();
  return total;
}

__global__ void __launch_bounds__(kScanThreads) bin_scan_kernel(const BinArgs A) {
  extern __shared__ int cnt[];  // counts, then offsets (padded layout)
  __shared__ int warp_tot[32];
  const int seg = blockIdx.x;
  int32_t* off = A.bin_off + int64_t(seg) * (KF_NBINS + 1);
  int32_t* cur = A.cursor + int64_t(seg) * KF_NBINS;
  const int tid = threadIdx.x;
  for (int b = tid; b < KF_NBINS; b += kScanThreads) cnt[pad_idx(b)] = off[b];  // coalesced
  __syncthreads();
  const int total = scan_bins(cnt, warp_tot);
  if (tid == 0) off[KF_NBINS] = total;
  for (int b = tid; b < KF_NBINS; b += kScanThreads) {  // coalesced
    const int o = cnt[pad_idx(b)];
    off[b] = o;
    cur[b] = o;
  }
}

// The unordered counting sort of one segment per block, its counts and
// cursors in shared memory (one launch for all segments): (1) every point of
// the segment adds one to its bin's count, (2) the block turns the counts
// into exclusive offsets (written to bin_off) and cursors, (3) every point
// takes the next slot of its bin.  The order inside a bin is that of the
// shared-memory atomics: for kf_tuning.bin_unordered, whose users do not
// depend on it.
// The points [p0, p1) of xyz ([3][stride]) of one segment, by the whole
// block, with cnt (KF_NBINS padded ints of shared memory) and warp_tot.
// FINE: the counting sort runs over the KF_NBINS_FINE sub-bins (cnt holds
// as many), whose starts go to fine_off, and the bin starts to `off` are
// those of the even sub-bins (a bin is two consecutive sub-bins).
template <bool FINE = false>
__device__ __forceinline__ void bin_one_segment(const float* xyz, int64_t stride, int64_t p0, int64_t p1,
                                                int32_t* off, int32_t* fine_off, float4* out_pts, int32_t* out_id,
                                                int32_t* out_seg, int seg, int* cnt, int* warp_tot) {
  constexpr int NB = FINE ? KF_NBINS_FINE : KF_NBINS;
  constexpr int NPHI = FINE ? KF_BIN_PHI_FINE : KF_BIN_PHI;
  const int tid = threadIdx.x;
  for (int b = tid; b < NB; b += kScanThreads) cnt[pad_idx(b)] = 0;
  __syncthreads();
  // the points in batches of kSegBatch a thread, their loads issued together
  constexpr int kSegBatch = 4;
  for (int64_t g0 = p0 + tid; g0 < p1; g0 += int64_t(kScanThreads) * kSegBatch) {
    float x[kSegBatch], y[kSegBatch], z[kSegBatch];
#pragma unroll
    for (int u = 0; u < kSegBatch; ++u) {
      const int64_t g = g0 + int64_t(u) * kScanThreads;
      if (g < p1) {
        x[u] = xyz[g];
        y[u] = xyz[stride + g];
        z[u] = xyz[2 * stride + g];
      }
    }
#pragma unroll
    for (int u = 0; u < kSegBatch; ++u) {
      const int64_t g = g0 + int64_t(u) * kScanThreads;
      if (g < p1) {
        const int b = bin_of<NPHI>(x[u], y[u], z[u]);
        atomicAdd(&cnt[pad_idx(b)], 1);
        // with points out (hits: their ids travel in .w), out_id is scratch:
        // it keeps each point's bin for the second pass
        if (out_pts) out_id[g] = b;
      }
    }
  }
  __syncthreads();
  const int total = scan_bins<NB>(cnt, warp_tot);
  if (tid == 0) off[KF_NBINS] = total;
  if constexpr (FINE) {
    if (tid == 0) fine_off[KF_NBINS_FINE] = total;
    for (int b = tid; b < KF_NBINS_FINE; b += kScanThreads) fine_off[b] = cnt[pad_idx(b)];  // coalesced
    for (int b = tid; b < KF_NBINS; b += kScanThreads) off[b] = cnt[pad_idx(2 * b)];
  } else {
    for (int b = tid; b < KF_NBINS; b += kScanThreads) off[b] = cnt[pad_idx(b)];  // coalesced
  }
  // every start read before the scatter below moves the cursors on
  __syncthreads();
  for (int64_t g0 = p0 + tid; g0 < p1; g0 += int64_t(kScanThreads) * kSegBatch) {
    float x[kSegBatch], y[kSegBatch], z[kSegBatch];
    int bins[kSegBatch];
#pragma unroll
    for (int u = 0; u < kSegBatch; ++u) {
      const int64_t g = g0 + int64_t(u) * kScanThreads;
      if (g < p1) {
        x[u] = xyz[g];
        y[u] = xyz[stride + g];
        z[u] = xyz[2 * stride + g];
        bins[u] = out_pts ? out_id[g] : 0;
      }
    }
#pragma unroll
    for (int u = 0; u < kSegBatch; ++u) {
      const int64_t g = g0 + int64_t(u) * kScanThreads;
      if (g < p1) {
        const int i = int(g - p0);
        if (out_pts) {  // the bin from the first pass; out_id stays scratch
          const int64_t q = p0 + atomicAdd(&cnt[pad_idx(bins[u])], 1);
          out_pts[q] = make_float4(x[u], y[u], z[u], __int_as_float(i));
          if (out_seg) out_seg[q] = seg;
        } else {
          const int64_t q = p0 + atomicAdd(&cnt[pad_idx(bin_of<NPHI>(x[u], y[u], z[u]))], 1);
          out_id[q] = i;
          if (out_seg) out_seg[q] = seg;
        }
      }
    }
  }
}

template <bool FINE>
__global__ void __launch_bounds__(kScanThreads) bin_segment_kernel(const BinArgs A) {
  extern __shared__ int cnt[];  // counts, then cursors (padded layout)
  __shared__ int warp_tot[32];
  const int seg = blockIdx.x;
  bin_one_segment<FINE>(A.xyz, A.stride, A.seg_off[seg], min(A.seg_off[seg + 1], A.stride),
                        A.bin_off + int64_t(seg) * (KF_NBINS + 1),
                        FINE ? A.fine_off + int64_t(seg) * (KF_NBINS_FINE + 1) : nullptr, A.out_pts, A.out_id,
                        A.out_seg, seg, cnt, warp_tot);
}

// The same over a table of segments of different point sets (the events a
// serving iteration prepares), one block per entry.
template <bool FINE>
__global__ void __launch_bounds__(kScanThreads) bin_segment_table_kernel(const BinSegment* table) {
  extern __shared__ int cnt[];
  __shared__ int warp_tot[32];
  const BinSegment& T = table[blockIdx.x];
  bin_one_segment<FINE>(T.xyz, T.stride, T.p0, T.p1, T.bin_off, T.fine_off, T.out_pts, T.out_id, nullptr, 0, cnt,
                        warp_tot);
}

__global__ void __launch_bounds__(kPointThreads) bin_scatter_kernel(const BinArgs A, int nseg) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; g < A.stride; g += stride) {
    const int s = segment_of(A.seg_off, nseg, g);
    if (s < 0) continue;
    const float x = A.xyz[g], y = A.xyz[A.stride + g], z = A.xyz[2 * A.stride + g];
    const int b = bin_of(x, y, z);
    const int64_t p0 = A.seg_off[s];
    const int i = int(g - p0);
    const int64_t q = p0 + atomicAdd(&A.cursor[int64_t(s) * KF_NBINS + b], 1);
    if (q >= A.stride) continue;  // only for malformed offsets
    A.out_id[q] = i;
    if (A.out_pts) A.out_pts[q] = make_float4(x, y, z, __int_as_float(i));
    if (A.out_seg) A.out_seg[q] = s;
  }
}

// deterministic order: insertion sort by id inside each bin
__global__ void __launch_bounds__(kPointThreads) bin_sort_kernel(const BinArgs A, int nseg) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= int64_t(nseg) * KF_NBINS) return;
  const int s = int(t / KF_NBINS), b = int(t % KF_NBINS);
  const int32_t* off = A.bin_off + int64_t(s) * (KF_NBINS + 1);
  const int64_t p0 = A.seg_off[s];
  int64_t beg = p0 + off[b], end = p0 + off[b + 1];
  if (end > A.stride) end = A.stride;
  for (int64_t u = beg + 1; u < end; ++u) {
    const int id = A.out_id[u];
    const float4 pt = A.out_pts ? A.out_pts[u] : make_float4(0.f, 0.f, 0.f, 0.f);
    int64_t v = u - 1;
    while (v >= beg && A.out_id[v] > id) {
      A.out_id[v + 1] = A.out_id[v];
      if (A.out_pts) A.out_pts[v + 1] = A.out_pts[v];
      --v;
    }
    A.out_id[v + 1] = id;
    if (A.out_pts) A.out_pts[v + 1] = pt;
  }
}

constexpr int kMaxDevices = 64;

// a kernel's shared-memory attributes, set once per device (the serving loop
// bins from several threads' calls; setting them again is harmless)
template <class K>
static cudaError_t segment_smem_attrs(K kernel, int smem, std::atomic<bool>* done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < kMaxDevices && done[dev].load(std::memory_order_acquire)) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  // the largest shared-memory carveout (a block takes 68 KB, or 135 KB with
  // the sub-bins; its 1024 threads' registers already leave room for one
  // block per SM)
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                             int(cudaSharedmemCarveoutMaxShared));
  if (e == cudaSuccess && dev >= 0 && dev < kMaxDevices) done[dev].store(true, std::memory_order_release);
  return e;
}

cudaError_t launch_bin_segment_table(const BinSegment* table, int n, bool fine, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  static std::atomic<bool> attr_set[kMaxDevices], fine_attr_set[kMaxDevices];
  if (fine) {
    cudaError_t e = segment_smem_attrs(bin_segment_table_kernel<true>, kFineSmem, fine_attr_set);
    if (e != cudaSuccess) return e;
    bin_segment_table_kernel<true><<<n, kScanThreads, kFineSmem, st>>>(table);
    return cudaGetLastError();
  }
  cudaError_t e = segment_smem_attrs(bin_segment_table_kernel<false>, kScanSmem, attr_set);
  if (e != cudaSuccess) return e;
  bin_segment_table_kernel<false><<<n, kScanThreads, kScanSmem, st>>>(table);
  return cudaGetLastError();
}

cudaError_t launch_bin_points(const BinArgs& a, int n_segments, cudaStream_t st) {
  if (n_segments <= 0) return cudaSuccess;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (a.unordered) {  // one launch, one block per segment
    static std::atomic<bool> seg_attr_set[kMaxDevices], fine_attr_set[kMaxDevices];
    if (a.fine_off) {
      e = segment_smem_attrs(bin_segment_kernel<true>, kFineSmem, fine_attr_set);
      if (e != cudaSuccess) return e;
      bin_segment_kernel<true><<<n_segments, kScanThreads, kFineSmem, st>>>(a);
      return cudaGetLastError();
    }
    e = segment_smem_attrs(bin_segment_kernel<false>, kScanSmem, seg_attr_set);
    if (e != cudaSuccess) return e;
    bin_segment_kernel<false><<<n_segments, kScanThreads, kScanSmem, st>>>(a);
    return cudaGetLastError();
  }
  if (a.fine_off) return cudaErrorInvalidValue;  // sub-bins only with the unordered binning
  e = cudaMemsetAsync(a.bin_off, 0, size_t(n_segments) * (KF_NBINS + 1) * sizeof(int32_t), st);
  if (e != cudaSuccess) return e;
  const int64_t pts = a.stride > 0 ? a.stride : 1;
  const int pgrid = int(std::min<int64_t>((pts + kPointThreads - 1) / kPointThreads, int64_t(1) << 20));
  bin_count_kernel<<<pgrid, kPointThreads, 0, st>>>(a, n_segments);
  // the scan kernel's shared-memory attribute, set once per device (the
  // serving loop bins point sets of many events; setting it again from
  // another thread is harmless, the value being the same)
  static std::atomic<bool> scan_attr_set[kMaxDevices];
  if (dev < 0 || dev >= kMaxDevices || !scan_attr_set[dev].load(std::memory_order_acquire)) {
    e = cudaFuncSetAttribute(bin_scan_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kScanSmem);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < kMaxDevices) scan_attr_set[dev].store(true, std::memory_order_release);
  }
  bin_scan_kernel<<<n_segments, kScanThreads, kScanSmem, st>>>(a);
  bin_scatter_kernel<<<pgrid, kPointThreads, 0, st>>>(a, n_segments);
  const int64_t bins = int64_t(n_segments) * KF_NBINS;
  if (!a.unordered)
    bin_sort_kernel<<<int((bins + kPointThreads - 1) / kPointThreads), kPointThreads, 0, st>>>(a, n_segments);
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
  if (out->fine_off && !ctx->tune.bin_unordered) return KF_EINVAL;  // sub-bins: unordered binning only
  out->n_events = in->n_events;
  out->n_layers = in->n_layers;
  out->first_layer = in->first_layer;
  out->n_hits = in->n_hits;
  out->seg_off = in->seg_off;
  const int nseg = in->n_events * in->n_layers;
  if (nseg == 0) return KF_OK;
  KF_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  const size_t id_bytes = (size_t(in->n_hits > 0 ? in->n_hits : 1) * sizeof(int32_t) + 255) & ~size_t(255);
  int rc = scratch_reserve(ctx, ctx->s_bin_id, id_bytes + size_t(nseg) * KF_NBINS * sizeof(int32_t));
  if (rc) return rc;
  BinArgs a;
  a.xyz = in->xyz;
  a.stride = in->n_hits;
  a.seg_off = in->seg_off;
  a.bin_off = out->bin_off;
  a.out_pts = reinterpret_cast<float4*>(out->hits);
  a.out_id = static_cast<int32_t*>(ctx->s_bin_id.ptr);
  a.out_seg = nullptr;
  a.cursor = reinterpret_cast<int32_t*>(static_cast<char*>(ctx->s_bin_id.ptr) + id_bytes);
  a.unordered = ctx->tune.bin_unordered;
  a.fine_off = out->fine_off;
  KF_CUDA_TRY(ctx, launch_bin_points(a, nseg, static_cast<cudaStream_t>(stream)));
  return KF_OK;
}
