// kf_build.cu -- combinatorial track building with the clone engine
// (Cerati et al., Sec. 3).
//
// Grouped layouts: one launch per building layer.  An 8-lane group of a warp
// owns one seed; lane k holds the seed's candidate of rank k (up to
// max_cands <= 8).  Per layer each live lane
//   1. propagates its candidate to the layer radius (kf::propagate),
//   2. derives the hit window: chi2 >= (u.r)^2 / (u^T S u) for every unit u,
//      so a hit with chi2 < cut lies within sqrt(cut u^T S u) of the
//      prediction along the tangent, the normal and z; those bounds, each
//      widened by 0.1 % plus 1e-6 rad / 1e-5 cm against rounding, are mapped
//      to eta x phi bins,
//   3. computes the chi2 increment of every hit in the window and keeps its
//      best children in a sorted register list (the bookkeeping list of the
//      clone engine: parent, hit, chi2_tot, nHits -- no state is copied),
//   4. the group merges its lanes' lists by shuffles into the seed's best
//      max_cands children, ranked by (nHits desc, chi2_tot asc, parent rank
//      asc, hit id asc), encoded as one 64-bit key,
//   5. only then are the winners materialised: lane k pulls the predicted
//      state of its parent by shuffles and applies the Kalman update with its
//      hit (a candidate with no compatible hit continues unchanged after
//      propagation).
// The hit history is kept as per-layer back-pointers (parent rank, hit id)
// and resolved once at the end, instead of copying index arrays per child.
// The candidate-packed step (below) computes the same per candidate with
// threads assigned to live candidates, and takes a block's seeds through
// several layers in one launch where the candidate buffers allow it.
#include "kf_bin.cuh"
#include "kf_build.cuh"
#include "kf_internal.h"
#include "kf_math.cuh"
#include "kf_tma.cuh"

#include <algorithm>
#include <climits>
#include <vector>

namespace kfi {

__device__ __forceinline__ uint64_t make_key(int nhits, float chi2tot, int parent, int hit_plus1) {
  return (uint64_t(255 - nhits) << 56) | (uint64_t(__float_as_uint(chi2tot)) << 24) | (uint64_t(parent) << 21) |
         uint64_t(hit_plus1);
}

// insert (key, pos) into the ascending list L/P (LW entries, last dropped)
template <int LW>
__device__ __forceinline__ void list_insert(uint64_t (&L)[LW], int (&P)[LW], uint64_t key, int pos) {
#pragma unroll
  for (int t = 0; t < LW; ++t) {
    if (key < L[t]) {
      const uint64_t tk = L[t];
      const int tp = P[t];
      L[t] = key;
      P[t] = pos;
      key = tk;
      pos = tp;
    }
  }
}

// Hit staging, per warp.  The four seeds of a warp are consecutive in
// (eta, phi) bin order, so their windows cluster: the warp takes the union of
// its candidates' windows (eta rows emin..emax; in phi the hull of the
// windows unwrapped around a reference bin, one or two bin ranges on the
// circle), stages the bin offsets of that hull in shared memory with plain
// loads and the hits of every (row, range) piece -- contiguous in the binned
// hit array -- with one bulk asynchronous copy each (cp.async.bulk, completed
// on the warp's mbarrier).  The chi2 scans then read shared memory only.  A
// warp whose hull does not fit, or whose seeds belong to more than one event,
// scans global memory.  Warps stage independently: no block-wide barrier.
// TILE (hits staged per warp; 0: no staging, every scan reads the L2-resident
// hits through L1), LW (entries of a lane's child list, >= max_cands) and
// COOP (the seed's lanes scan each parent's window together, instead of each
// lane its own candidate's) are launch parameters picked by the autotuner.
constexpr int kWarps = kBuildThreads / 32;
constexpr int kStageOffs = 384;  // bin offsets staged per warp
constexpr int kStagePieces = 2 * KF_BIN_ETA;
constexpr uint32_t kBuildWaitLimit = 1u << 22;  // bounded mbarrier polls

__device__ __forceinline__ int wrap_phi(int d) {  // to [-KF_BIN_PHI/2, KF_BIN_PHI/2)
  return ((d + KF_BIN_PHI / 2) & (KF_BIN_PHI - 1)) - KF_BIN_PHI / 2;
}

// Window of a predicted candidate: S^-1 = (C_pos + V)^-1, and the eta rows
// e0..e1 and phi bins fa0..fa1, fb0..fb1 (second part when the window wraps
// around phi = +-pi) that can hold a hit with chi2 < cut at radius R; the
// phi bins are those of a row of nphi bins over [-pi, pi) (KF_BIN_PHI, or
// KF_BIN_PHI_FINE for the sub-bins), fa1 preset by the caller to nphi - 1.
__device__ __forceinline__ void hit_window(const float p[6], const float lo[3], const float C[21], float R, float v0,
                                           float v1, float v2, float cut, float Si[6], int& e0, int& e1, int& fa0,
                                           int& fa1, int& fb0, int& fb1, int nphi = KF_BIN_PHI) {
  kf::inverse_S(C, v0, v1, v2, Si);
  const float X = p[0] + lo[0], Y = p[1] + lo[1], Z = p[2] + lo[2];
  // direction cosines of the position: they only scale the widths below,
  // which are widened by 0.1 %, so a reciprocal square root is exact enough
  const float irr = rsqrtf(X * X + Y * Y);
  const float cph = X * irr, sph = Y * irr;
  const float s00 = C[0] + v0, s10 = C[1], s11 = C[2] + v1, s22 = C[5] + v2;
  const float Stt = sph * sph * s00 - 2.f * sph * cph * s10 + cph * cph * s11;
  const float Snn = cph * cph * s00 + 2.f * sph * cph * s10 + sph * sph * s11;
  const float wt = sqrtf(cut * fmaxf(Stt, 0.f));
  const float wn = sqrtf(cut * fmaxf(Snn, 0.f));
  const float wz = sqrtf(cut * fmaxf(s22, 0.f));
  // A hit with chi2 < cut lies within wt of the prediction along the tangent,
  // wn along the normal and wz in z (chi2 >= (u.r)^2 / u^T S u for any unit
  // u), so its distance from the axis is between R - wn and
  // sqrt((R + wn)^2 + wt^2) and its phi within atan(wt / (R - wn)) of the
  // prediction's.  The bounds are widened by 0.1 % plus a small absolute
  // term -- far above the float rounding of the window, of the chi2 and of
  // the hits' own bins -- and cover exactly the bins they reach; the phi
  // half-width takes atan(x) <= x (x >= 0), a bound from above.
  constexpr float kWiden = 1.001f;
  const float rin = R - wn * kWiden;
  const float phic = atan2f(Y, X);
  const float dphi = (rin > 0.5f * R && wt * kWiden < rin) ? (wt * kWiden / rin) * kWiden + 1e-6f : 10.f;
  if (dphi < 1.f && phic >= -kPi && phic <= kPi) {  // also false for NaN
    // the sub-bin scale is exactly twice the bin scale (a power of two), so a
    // hit's sub-bin halved is its bin
    const float scale = float(nphi) / (2.0f * kPi);
    const int f0 = __float2int_rd((phic - dphi + kPi) * scale);
    const int f1 = __float2int_rd((phic + dphi + kPi) * scale);
    if (f1 - f0 + 1 < nphi) {
      if (f0 < 0) {
        fa0 = f0 + nphi;
        fb0 = 0;
        fb1 = f1;
      } else if (f1 >= nphi) {
        fa0 = f0;
        fb0 = 0;
        fb1 = f1 - nphi;
      } else {
        fa0 = f0;
        fa1 = f1;
      }
    }
  }
  // eta bins: z within Z +- wz over the hit radii above
  e0 = 0;
  e1 = KF_BIN_ETA - 1;
  const float rlo = R - wn * kWiden - 1e-5f;
  const float rhi = sqrtf((R + wn) * (R + wn) + wt * wt) * kWiden + 1e-5f;
  if (rlo > 0.f) {
    const float zlo = Z - wz * kWiden - 1e-5f, zhi = Z + wz * kWiden + 1e-5f;
    const float tmin = zlo >= 0.f ? zlo / rhi : zlo / rlo;
    const float tmax = zhi >= 0.f ? zhi / rlo : zhi / rhi;
    // asinh by log(|t| + sqrt(t^2 + 1)) with the fast logarithm, widened by
    // 1e-5 in eta (far above that form's error): still a superset
    e0 = eta_bin(copysignf(__logf(fabsf(tmin) + sqrtf(fmaf(tmin, tmin, 1.f))), tmin) - 1e-5f);
    e1 = eta_bin(copysignf(__logf(fabsf(tmax) + sqrtf(fmaf(tmax, tmax, 1.f))), tmax) + 1e-5f);
  }
}

// Clone engine, one seed per 8-lane group: the lanes' sorted child lists
// (L, P) are merged by shuffles into the seed's best max_cands keys.  Lane k
// receives the k-th best (key, parent rank, hit position); every lane gets
// the number of children kept.
template <int LW>
__device__ __forceinline__ void merge_group(uint64_t (&L)[LW], int (&P)[LW], int max_cands, int k, int gbase,
                                            uint64_t& my_key, int& my_parent, int& my_pos, int& n_win) {
#pragma unroll
  for (int r = 0; r < LW; ++r) {
    if (r < max_cands) {  // uniform over the launch; max_cands <= LW
      uint64_t m = L[0];
#pragma unroll
      for (int d = kGroup / 2; d >= 1; d >>= 1) {
        const uint64_t o = __shfl_xor_sync(kFull, m, d);
        m = o < m ? o : m;
      }
      const bool mine = (L[0] == m) && (m != kNoKey);
      const unsigned bal = (__ballot_sync(kFull, mine) >> gbase) & 0xffu;
      const int wl = bal ? __ffs(bal) - 1 : 0;
      const int wpos = __shfl_sync(kFull, P[0], gbase + wl);
      if (mine) {
#pragma unroll
        for (int t = 0; t < LW - 1; ++t) {
          L[t] = L[t + 1];
          P[t] = P[t + 1];
        }
        L[LW - 1] = kNoKey;
        P[LW - 1] = -1;
      }
      if (m != kNoKey) {
        if (k == r) {
          my_key = m;
          my_parent = int((m >> 21) & 7u);
          my_pos = wpos;
        }
        ++n_win;
      }
    }
  }
}

// Five blocks of 128 threads per SM (20 warps, at most 96 registers): more
// resident warps hide the dependent loads of the window scans better than
// the spills they cost (measured: 3.43 vs 3.78 ms per 7-layer build at N = 6).
template <int TILE, int LW, bool COOP>
__global__ void __launch_bounds__(kBuildThreads, kBuildBlocksPerSM) build_step_kernel(const BuildStepArgs Args) {
  extern __shared__ float4 s_hits_all[];
  __shared__ BuildSlot sD;
  __shared__ int32_t s_off_all[TILE > 0 ? kWarps : 1][TILE > 0 ? kStageOffs : 1];
  __shared__ int s_pob_all[TILE > 0 ? kWarps : 1][TILE > 0 ? kStagePieces : 1];  // per piece: offset base
  __shared__ int s_phb_all[TILE > 0 ? kWarps : 1][TILE > 0 ? kStagePieces : 1];  // per piece: hit base
  __shared__ int s_stage_all[kWarps];
  __shared__ __align__(8) uint64_t s_bar_all[kWarps];
  const int warp = threadIdx.x >> 5;
  float4* const s_hits = s_hits_all + warp * TILE;
  int32_t* const s_off = s_off_all[TILE > 0 ? warp : 0];
  int* const s_pob = s_pob_all[TILE > 0 ? warp : 0];
  int* const s_phb = s_phb_all[TILE > 0 ? warp : 0];
  uint64_t* const s_bar = &s_bar_all[warp];
  if (threadIdx.x == 0) {
    int sl = 0;
    while (sl + 1 < Args.n_slots && int(blockIdx.x) >= Args.slots[sl + 1].block_begin) ++sl;
    sD = Args.slots[sl];
  }
  if (TILE > 0 && (threadIdx.x & 31) == 0) {
    mbar_init(s_bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  const BuildSlot& D = sD;
  const int lane = threadIdx.x & 31;
  const int k = lane & (kGroup - 1);
  const int gbase = lane & ~(kGroup - 1);
  const int64_t j = (int64_t(blockIdx.x - D.block_begin) * kBuildThreads + threadIdx.x) / kGroup;
  const int64_t S8 = D.S * kGroup;
  const bool seed_ok = j < D.S;
  const int nc = seed_ok ? D.in.ncand[j] : 0;
  const bool active = k < nc;
  const int64_t slot = cand_slot(j, k, D.S, D.in_rm), oslot = cand_slot(j, k, D.S, D.out_rm);

  float p[6], lo[3], C[21];
  float chi2tot = 0.f;
  int nh = 0;
  int32_t st = 0;
  if (active) {
#pragma unroll
    for (int c = 0; c < 6; ++c) p[c] = D.in.par[c * S8 + slot];
#pragma unroll
    for (int c = 0; c < 3; ++c) lo[c] = D.in.par[(6 + c) * S8 + slot];
#pragma unroll
    for (int c = 0; c < 21; ++c) C[c] = D.in.cov[c * S8 + slot];
    chi2tot = D.in.chi2[slot];
    const int32_t meta = D.in.meta[slot];
    nh = meta & 0xff;
    st = meta >> 8;
  } else {
#pragma unroll
    for (int c = 0; c < 6; ++c) p[c] = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) lo[c] = 0.f;
#pragma unroll
    for (int c = 0; c < 21; ++c) C[c] = 0.f;
  }
  const int e = seed_ok ? (D.seed_evt ? D.seed_evt[j] : 0) : 0;
  const float a = Args.a_scale * (seed_ok ? float(D.charge[D.seed_perm[j]]) : 1.f);
  const int seg = e * D.n_layers + D.layer;
  const int64_t h0 = seed_ok ? D.seg_off[seg] : 0;
  bool stopped = (st & KF_ST_STOPPED) != 0;
  if (active && !stopped) {
    const int r = kf::propagate<float, kNewtonBuild, true>(p, lo, C, a, D.R);
    if (r) {
      st |= r;
      stopped = true;
    } else if (D.x_x0 > 0.f) {
      kf::scatter(p, lo, C, D.x_x0, Args.mass);
    }
  }

  // ---- hit window of this candidate: eta rows e0..e1, phi bins fa0..fa1
  // and fb0..fb1 (second part when the window wraps around phi = +-pi)
  const bool scan = active && !stopped;
  float Si[6];
  int e0 = 0, e1 = -1, fa0 = 0, fa1 = KF_BIN_PHI - 1, fb0 = 0, fb1 = -1;
  if (scan) hit_window(p, lo, C, D.R, Args.v0, Args.v1, Args.v2, Args.cut, Si, e0, e1, fa0, fa1, fb0, fb1);
  const int32_t* boff = D.bin_off + int64_t(seg) * (KF_NBINS + 1);

  // ---- warp union of the windows and staging (TILE > 0)
  bool staged = false, timed_out = false;
  bool armed = false;  // (lane 0) copies issued into this warp's tile
  int emin = 0, hs0a = 0, hs1a = KF_BIN_PHI - 1, hs1b = -1;
  if constexpr (TILE > 0) {
    // phi unwrapped around the bin of the warp's first seed; any reference is
    // correct, a near one keeps the hull small
    const int64_t j_first = j - (lane >> 3);
    int f_ref = 0;
    if (j_first < D.S) {
      const int64_t s0 = cand_slot(j_first, 0, D.S, D.in_rm);
      const float ph = atan2f(D.in.par[S8 + s0], D.in.par[s0]);
      if (ph >= -kPi && ph <= kPi) f_ref = phi_bin(ph);
    }
    int d0 = KF_BIN_PHI, d1 = -KF_BIN_PHI;
    if (scan) {
      d0 = wrap_phi(fa0 - f_ref);
      d1 = fb1 >= fb0 ? d0 + (KF_BIN_PHI - fa0) + fb1  // wrapped: fa0..255 then 0..fb1
                      : d0 + (fa1 - fa0);
    }
    emin = __reduce_min_sync(kFull, scan ? e0 : KF_BIN_ETA);
    const int emax = __reduce_max_sync(kFull, scan ? e1 : -1);
    const int umin = __reduce_min_sync(kFull, d0), umax = __reduce_max_sync(kFull, d1);
    const int segmin = __reduce_min_sync(kFull, scan ? seg : INT_MAX);
    const int segmax = __reduce_max_sync(kFull, scan ? seg : -1);
    // the hull: phi bins hs0a..hs1a and 0..hs1b (empty if hs1b < 0)
    if (umax - umin + 1 < KF_BIN_PHI) {
      const int fh = (f_ref + umin + 2 * KF_BIN_PHI) & (KF_BIN_PHI - 1), W = umax - umin + 1;
      hs0a = fh;
      hs1a = min(fh + W - 1, KF_BIN_PHI - 1);
      hs1b = fh + W - 1 - KF_BIN_PHI;
    }
    const int nrows = emax - emin + 1;
    staged = nrows > 0 && segmin == segmax;
    if (staged) {
      const int lena = hs1a - hs0a + 2, lenb = hs1b + 2;  // offsets per piece (bins + end)
      const int per_row = lena + (lenb >= 2 ? lenb : 0);
      staged = nrows * per_row <= kStageOffs;
      if (staged) {
        // bin offsets of every piece, then the piece table and the copies
        for (int q = 0; q < 2 * nrows; ++q) {
          const int len = (q & 1) ? lenb : lena;
          if (len < 2) continue;
          const int32_t* src = boff + (emin + (q >> 1)) * KF_BIN_PHI + ((q & 1) ? 0 : hs0a);
          const int ob = (q >> 1) * per_row + ((q & 1) ? lena : 0);
          for (int t = lane; t < len; t += 32) s_off[ob + t] = src[t];
        }
        __syncwarp();
        if (lane == 0) {
          int nh_tot = 0;
          for (int q = 0; q < 2 * nrows; ++q) {
            const int len = (q & 1) ? lenb : lena;
            const int ob = (q >> 1) * per_row + ((q & 1) ? lena : 0);
            s_pob[q] = ob;
            s_phb[q] = nh_tot;
            if (len >= 2) nh_tot += s_off[ob + len - 1] - s_off[ob];
          }
          int st_flag = nh_tot <= TILE ? 1 : 0;
          // test hook: this warp issues nothing, so its wait below runs out
          const bool skip = (int64_t(blockIdx.x) * kBuildThreads + threadIdx.x) / 32 == Args.test_skip_warp;
          if (st_flag && nh_tot > 0 && skip) {
            st_flag = 2;
          } else if (st_flag && nh_tot > 0) {
            armed = true;
            mbar_arrive_expect_tx(s_bar, uint32_t(nh_tot) * uint32_t(sizeof(float4)));
            for (int q = 0; q < 2 * nrows; ++q) {
              const int len = (q & 1) ? lenb : lena;
              if (len < 2) continue;
              const int u0 = s_off[s_pob[q]], cnt = s_off[s_pob[q] + len - 1] - u0;
              if (cnt > 0)
                bulk_g2s(s_hits + s_phb[q], D.hits + h0 + u0, uint32_t(cnt) * uint32_t(sizeof(float4)), s_bar);
            }
            st_flag = 2;  // copies in flight
          }
          s_stage_all[warp] = st_flag;
        }
        __syncwarp();
        const int flag = s_stage_all[warp];
        staged = flag != 0;
        const uint32_t limit = Args.test_wait_limit ? Args.test_wait_limit : kBuildWaitLimit;
        if (flag == 2 && !mbar_wait_bounded(s_bar, 0, limit)) {
          // a copy did not complete: stop the warp's candidates with the error bit
          st |= KF_ST_DEVICE_TIMEOUT;
          stopped = true;
        }
      }
    }
    timed_out = __any_sync(kFull, stopped && (st & KF_ST_DEVICE_TIMEOUT));
  }

  // ---- bookkeeping list of this parent's children (keys only)
  uint64_t L[LW];
  int P[LW];
#pragma unroll
  for (int t = 0; t < LW; ++t) {
    L[t] = kNoKey;
    P[t] = -1;
  }
  if constexpr (!COOP) {
    // each lane scans the window of its own candidate
    if (active) {
      bool any = false;
      if (!stopped) {
        for (int er = e0; er <= e1; ++er) {
          for (int part = 0; part < 2; ++part) {
            const int f0 = part == 0 ? fa0 : fb0, f1 = part == 0 ? fa1 : fb1;
            if (f1 < f0) continue;
            // the piece of the staged hull holding f0..f1 (always one of the
            // two when staged; checked all the same)
            const int pc = (f0 >= hs0a && f1 <= hs1a) ? 0 : 1;
            const int ph0 = pc ? 0 : hs0a, ph1 = pc ? hs1b : hs1a;
            const bool in_smem = TILE > 0 && staged && f0 >= ph0 && f1 <= ph1;
            int u0, u1, ubias = 0;
            const float4* hs = D.hits + h0;
            if (in_smem) {
              const int q = 2 * (er - emin) + pc;
              const int32_t* off = s_off + (s_pob[q] - ph0);
              u0 = off[f0];
              u1 = off[f1 + 1];
              hs = s_hits;
              ubias = s_phb[q] - s_off[s_pob[q]];
            } else {
              u0 = boff[er * KF_BIN_PHI + f0];
              u1 = boff[er * KF_BIN_PHI + f1 + 1];
            }
            for (int u = u0; u < u1; ++u) {
              const float4 m = hs[u + ubias];
              const float r0 = (m.x - p[0]) - lo[0], r1 = (m.y - p[1]) - lo[1], r2 = (m.z - p[2]) - lo[2];
              const float c2 = kf::chi2_of(r0, r1, r2, Si);
              if (c2 < Args.cut) {
                const int id = __float_as_int(m.w);
                if (id < KF_MAX_HITS_PER_SEGMENT) {
                  list_insert(L, P, make_key(nh + 1, chi2tot + c2, k, id + 1), u);
                  any = true;
                }
              }
            }
          }
        }
      }
      // no compatible hit (or a stopped candidate): one child without a hit
      if (!any) list_insert(L, P, make_key(nh, chi2tot, k, 0), -1);
    }
  } else {
    // The seed's lanes scan together: for each parent c in turn, its
    // prediction, S^-1 and window are broadcast to the group and the 8 lanes
    // take the window's hits with stride 8, each inserting the children it
    // finds into its own list (the key carries the parent).  Any key of the
    // seed's best max_cands is among the best max_cands of the lane holding it,
    // so the merge below is unchanged; the keys are a total order, so the
    // result does not depend on which lane scanned which hit.
    const bool scan_me = active && !stopped;
    if (!scan_me) {
  #pragma unroll
      for (int c = 0; c < 6; ++c) Si[c] = 0.f;
    }
    bool any_mine = false;  // a compatible hit was found for this lane's candidate
  #pragma unroll 1
    for (int c = 0; c < Args.max_cands; ++c) {
      const int src = gbase + c;
      const bool cs = __shfl_sync(kFull, int(scan_me), src) != 0;
      const float q0 = __shfl_sync(kFull, p[0], src), q1 = __shfl_sync(kFull, p[1], src),
                  q2 = __shfl_sync(kFull, p[2], src);
      const float l0 = __shfl_sync(kFull, lo[0], src), l1 = __shfl_sync(kFull, lo[1], src),
                  l2 = __shfl_sync(kFull, lo[2], src);
      float cSi[6];
  #pragma unroll
      for (int t = 0; t < 6; ++t) cSi[t] = __shfl_sync(kFull, Si[t], src);
      const int ce0 = __shfl_sync(kFull, e0, src), ce1 = __shfl_sync(kFull, e1, src);
      const int cfa0 = __shfl_sync(kFull, fa0, src), cfa1 = __shfl_sync(kFull, fa1, src);
      const int cfb0 = __shfl_sync(kFull, fb0, src), cfb1 = __shfl_sync(kFull, fb1, src);
      const int cnh = __shfl_sync(kFull, nh, src);
      const float cchi = __shfl_sync(kFull, chi2tot, src);
      bool found = false;
      if (cs) {
        for (int er = ce0; er <= ce1; ++er) {
          for (int part = 0; part < 2; ++part) {
            const int f0 = part == 0 ? cfa0 : cfb0, f1 = part == 0 ? cfa1 : cfb1;
            if (f1 < f0) continue;
            // the piece of the staged hull holding f0..f1 (always one of the
            // two when staged; checked all the same)
            const int pc = (f0 >= hs0a && f1 <= hs1a) ? 0 : 1;
            const int ph0 = pc ? 0 : hs0a, ph1 = pc ? hs1b : hs1a;
            const bool in_smem = TILE > 0 && staged && f0 >= ph0 && f1 <= ph1;
            int u0, u1, ubias = 0;
            const float4* hs = D.hits + h0;
            if (in_smem) {
              const int q = 2 * (er - emin) + pc;
              const int32_t* off = s_off + (s_pob[q] - ph0);
              u0 = off[f0];
              u1 = off[f1 + 1];
              hs = s_hits;
              ubias = s_phb[q] - s_off[s_pob[q]];
            } else {
              u0 = boff[er * KF_BIN_PHI + f0];
              u1 = boff[er * KF_BIN_PHI + f1 + 1];
            }
            for (int u = u0 + k; u < u1; u += kGroup) {
              const float4 m = hs[u + ubias];
              const float r0 = (m.x - q0) - l0, r1 = (m.y - q1) - l1, r2 = (m.z - q2) - l2;
              const float c2 = kf::chi2_of(r0, r1, r2, cSi);
              if (c2 < Args.cut) {
                const int id = __float_as_int(m.w);
                if (id < KF_MAX_HITS_PER_SEGMENT) {
                  list_insert(L, P, make_key(cnh + 1, cchi + c2, c, id + 1), u);
                  found = true;
                }
              }
            }
          }
        }
      }
      const unsigned fb = (__ballot_sync(kFull, found) >> gbase) & 0xffu;
      if (k == c) any_mine = fb != 0;
    }
    // no compatible hit (or a stopped candidate): one child without a hit
    if (active && !any_mine) list_insert(L, P, make_key(nh, chi2tot, k, 0), -1);
  }
  // nothing in flight at exit: after a timeout, lane 0 waits (bounded) for the
  // copies it issued, if it issued any
  if (TILE > 0 && timed_out && lane == 0 && armed) mbar_wait_bounded(s_bar, 0, kBuildWaitLimit);

  // ---- clone engine: merge the group's lists into the best max_cands
  uint64_t my_key = kNoKey;
  int my_parent = 0, my_pos = -1, n_win = 0;
  merge_group(L, P, Args.max_cands, k, gbase, my_key, my_parent, my_pos, n_win);

  // ---- materialise the winners: pull the parent's predicted state
  const int src = gbase + my_parent;
  float q[6], ql[3], qC[21];
#pragma unroll
  for (int c = 0; c < 6; ++c) q[c] = __shfl_sync(kFull, p[c], src);
#pragma unroll
  for (int c = 0; c < 3; ++c) ql[c] = __shfl_sync(kFull, lo[c], src);
#pragma unroll
  for (int c = 0; c < 21; ++c) qC[c] = __shfl_sync(kFull, C[c], src);
  const int32_t pst = __shfl_sync(kFull, st, src);
  const int pstopped = __shfl_sync(kFull, int(stopped), src);
  if (seed_ok && k < n_win) {
    const int nh_new = 255 - int(my_key >> 56);
    const float chi2_new = __uint_as_float(uint32_t(my_key >> 24));
    const int hit_plus1 = int(my_key & 0x1fffffu);
    int32_t st_new = pst;
    if (hit_plus1 > 0) {
      const float4 m = D.hits[h0 + my_pos];
      float Si[6];
      kf::inverse_S(qC, Args.v0, Args.v1, Args.v2, Si);
      float r0, r1, r2;
      kf::residual<float, true>(q, ql, m.x, m.y, m.z, r0, r1, r2);
      kf::kalman_update<float, true>(q, ql, qC, Si, r0, r1, r2, Args.v0, Args.v1, Args.v2);
    } else if (!pstopped) {
      st_new |= KF_ST_NO_HIT;
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) D.out.par[c * S8 + oslot] = q[c];
#pragma unroll
    for (int c = 0; c < 3; ++c) D.out.par[(6 + c) * S8 + oslot] = ql[c];
#pragma unroll
    for (int c = 0; c < 21; ++c) D.out.cov[c * S8 + oslot] = qC[c];
    D.out.chi2[oslot] = chi2_new;
    D.out.meta[oslot] = nh_new | (st_new << 8);
    D.hist_parent[oslot] = int8_t(my_parent);
    D.hist_hit[oslot] = hit_plus1 - 1;
  }
  if (seed_ok && k == 0) D.out.ncand[j] = int8_t(n_win);
}

// Chi2 scan of one predicted candidate's window (one thread): rows e0..e1,
// each the hits of bins fa0..fa1 then fb0..fb1 of the segment's binned hits
// `hs` (bin offsets `boff`, nphi of them a row); the next row's bin offsets and the next hit are
// loaded one step ahead.  Every hit with chi2 < cut (and an id below the
// segment limit) becomes a child key (nh + 1, chi2tot + chi2, parent rank k,
// id + 1) in the sorted list (L, P).  Returns whether any hit was compatible.
template <int LW>
__device__ __forceinline__ bool scan_window(const float p[6], const float lo[3], const float Si[6], int e0, int e1,
                                            int fa0, int fa1, int fb0, int fb1, const int32_t* boff,
                                            const float4* hs, float cut, int nh, float chi2tot, int k,
                                            uint64_t (&L)[LW], int (&P)[LW], int nphi = KF_BIN_PHI) {
  bool any = false;
  const bool two = fb1 >= fb0;
  int na0 = 0, na1 = 0, nb0 = 0, nb1 = 0;
  if (e0 <= e1) {
    const int32_t* q = boff + e0 * nphi;
    na0 = q[fa0];
    na1 = q[fa1 + 1];
    if (two) {
      nb0 = q[fb0];
      nb1 = q[fb1 + 1];
    }
  }
  for (int er = e0; er <= e1; ++er) {
    const int a0 = na0, na = na1 - na0, b0 = nb0, n = na + (nb1 - nb0);
    if (er < e1) {
      const int32_t* q = boff + (er + 1) * nphi;
      na0 = q[fa0];
      na1 = q[fa1 + 1];
      if (two) {
        nb0 = q[fb0];
        nb1 = q[fb1 + 1];
      }
    }
    float4 mn = make_float4(0.f, 0.f, 0.f, 0.f);
    if (n > 0) mn = hs[na > 0 ? a0 : b0];
    for (int v = 0; v < n; ++v) {
      const int u = v < na ? a0 + v : b0 + (v - na);
      const float4 m = mn;
      if (v + 1 < n) mn = hs[v + 1 < na ? a0 + v + 1 : b0 + (v + 1 - na)];
      const float r0 = (m.x - p[0]) - lo[0], r1 = (m.y - p[1]) - lo[1], r2 = (m.z - p[2]) - lo[2];
      const float c2 = kf::chi2_of(r0, r1, r2, Si);
      if (c2 < cut) {
        const int id = __float_as_int(m.w);
        if (id < KF_MAX_HITS_PER_SEGMENT) {
          list_insert(L, P, make_key(nh + 1, chi2tot + c2, k, id + 1), u);
          any = true;
        }
      }
    }
  }
  return any;
}

// The same scan with a row's hits loaded kScanBatch at a time: all loads of a
// batch are in flight before the first chi2 (the scan is bound by the round
// trips of its dependent loads, not by its arithmetic).  Used by the
// register-resident step: batches of 4 with one lane a seed, of 2 otherwise
// (where the registers are needed elsewhere).

template <int LW, int kScanBatch = 4>
__device__ __forceinline__ bool scan_window_batched(const float p[6], const float lo[3], const float Si[6], int e0, int e1,
                                            int fa0, int fa1, int fb0, int fb1, const int32_t* boff,
                                            const float4* hs, float cut, int nh, float chi2tot, int k,
                                            uint64_t (&L)[LW], int (&P)[LW], int nphi = KF_BIN_PHI) {
  bool any = false;
  const bool two = fb1 >= fb0;
  int na0 = 0, na1 = 0, nb0 = 0, nb1 = 0;
  if (e0 <= e1) {
    const int32_t* q = boff + e0 * nphi;
    na0 = q[fa0];
    na1 = q[fa1 + 1];
    if (two) {
      nb0 = q[fb0];
      nb1 = q[fb1 + 1];
    }
  }
  for (int er = e0; er <= e1; ++er) {
    const int a0 = na0, na = na1 - na0, b0 = nb0, n = na + (nb1 - nb0);
    if (er < e1) {
      const int32_t* q = boff + (er + 1) * nphi;
      na0 = q[fa0];
      na1 = q[fa1 + 1];
      if (two) {
        nb0 = q[fb0];
        nb1 = q[fb1 + 1];
      }
    }
    // the row's hits in batches of kScanBatch loads in flight
    for (int v0 = 0; v0 < n; v0 += kScanBatch) {
      float4 mb[kScanBatch];
      int ub[kScanBatch];
#pragma unroll
      for (int i = 0; i < kScanBatch; ++i) {
        const int v = v0 + i;
        ub[i] = v < na ? a0 + v : b0 + (v - na);
        if (v < n) mb[i] = hs[ub[i]];
      }
#pragma unroll
      for (int i = 0; i < kScanBatch; ++i) {
        if (v0 + i < n) {
          const float4 m = mb[i];
          const float r0 = (m.x - p[0]) - lo[0], r1 = (m.y - p[1]) - lo[1], r2 = (m.z - p[2]) - lo[2];
          const float c2 = kf::chi2_of(r0, r1, r2, Si);
          if (c2 < cut) {
            const int id = __float_as_int(m.w);
            if (id < KF_MAX_HITS_PER_SEGMENT) {
              list_insert(L, P, make_key(nh + 1, chi2tot + c2, k, id + 1), ub[i]);
              any = true;
            }
          }
        }
      }
    }
  }
  return any;
}

// ---- candidate-packed step (scan scheme 2)
//
// The same computation as build_step_kernel, with threads assigned to live
// candidates instead of fixed 8-lane seed groups.  A block serves 128 seeds
// (kPackSeeds; scheme 3: 64) in rounds; a round takes the next seeds whose
// parents fit the block's threads and runs three phases separated by block
// barriers:
//   1. the round's parents, packed onto consecutive threads, each propagate
//      their candidate, derive the window, scan it (global memory) and leave
//      the prediction and the sorted child list in shared memory;
//   2. one thread per seed merges its parents' lists into the best max_cands
//      keys -- the same selection as merge_group: the keys are a total order;
//   3. the kept children, packed the same way, are each updated with their hit
//      from the parent's prediction in shared memory and stored.
// In the early building layers a seed holds one or two candidates, where the
// grouped layout leaves most lanes of a warp idle through the propagation,
// the scan and the update; packed, every phase keeps the warps full.  Each
// candidate and child goes through the same functions as in the grouped
// step, so the results are bitwise equal.
constexpr int kStateWords = kParN + 21;  // x y z px py pz, lo x y z, covariance
constexpr int kStoppedBit = 1 << 30;     // parent stopped (status word in shared memory)

// Exclusive scan over the block's threads: start[0] = 0, start[t + 1] =
// start[t] + v of thread t.  All threads call; ends with a barrier.
template <int NT>
__device__ __forceinline__ void block_scan(int v, int* start, int* warp_sum) {
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  int x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int y = __shfl_up_sync(kFull, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) warp_sum[w] = x;
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NT / 32; ++q)
    if (q < w) x += warp_sum[q];
  start[t + 1] = x;
  if (t == 0) start[0] = 0;
  __syncthreads();
}

// The largest s in [lo, hi] with start[s] <= v.
__device__ __forceinline__ int packed_owner(const int* start, int lo, int hi, int v) {
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (start[mid] <= v)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// NT threads per block, one seed per thread: 128 (5 blocks per SM) or 64 (10
// blocks per SM: a block barrier holds two warps, not four); 20 warps per SM
// either way, at most 96 registers.
template <int LW, int NT>
__global__ void __launch_bounds__(NT, kBuildBlocksPerSM * kBuildThreads / NT) build_step_packed_kernel(const BuildStepArgs Args) {
  __shared__ BuildSlot sD;
  __shared__ float s_state[kStateWords][NT];  // the round's parent predictions
  __shared__ uint64_t s_key[LW][NT];          // and their sorted child lists
  __shared__ int s_pos[LW][NT];
  __shared__ int s_pst[NT];         // parent status | kStoppedBit
  __shared__ uint64_t s_ckey[NT][LW];  // kept children of the round's seeds, by rank
  __shared__ int s_cpos[NT][LW];
  __shared__ int s_pstart[NT + 1];  // parents of the block's seeds (exclusive scan)
  __shared__ int s_cstart[NT + 1];  // kept children of the round's seeds (exclusive scan)
  __shared__ int s_wsum[NT / 32];
  __shared__ float s_a[NT];      // per seed: a = c Bz q
  __shared__ int s_seg[NT];      // per seed: hit segment (event, layer)
  __shared__ int64_t s_h0[NT];   // per seed: first hit of the segment
  const int t = threadIdx.x;
  // one layer step, or (Args.layers > 1) every layer of the batch in turn for
  // the block's seeds: a seed's candidates are read and written by its block
  // only, so the block needs no other block between its layers
  const int n_steps = Args.layers > 1 ? Args.layers : 1;
  for (int li = 0; li < n_steps; ++li) {
  if (t == 0) {
    if (Args.layers > 1) {
      sD = Args.slots[li];
    } else {
      int sl = 0;
      while (sl + 1 < Args.n_slots && int(blockIdx.x) >= Args.slots[sl + 1].block_begin) ++sl;
      sD = Args.slots[sl];
    }
  }
  __syncthreads();
  const BuildSlot& D = sD;
  const int64_t S8 = D.S * kGroup;
  const int spb = Args.pack_seeds > 0 && Args.pack_seeds < NT ? Args.pack_seeds : NT;
  const int64_t j0 = int64_t(blockIdx.x - D.block_begin) * spb;
  const int ns = int(D.S - j0 < spb ? D.S - j0 : spb);
  if (t < ns) {  // per-seed constants, read once (visible after the scan's barriers)
    const int64_t j = j0 + t;
    const int seg = (D.seed_evt ? D.seed_evt[j] : 0) * D.n_layers + D.layer;
    s_seg[t] = seg;
    s_h0[t] = D.seg_off[seg];
    s_a[t] = Args.a_scale * float(D.charge[D.seed_perm[j]]);
  }
  block_scan<NT>(t < ns ? int(D.in.ncand[j0 + t]) : 0, s_pstart, s_wsum);

  for (int sa = 0; sa < ns;) {  // uniform over the block
    // the round: seeds [sa, sb), parents s_pstart[sa] .. s_pstart[sb] - 1
    const int base = s_pstart[sa];
    const int sb = packed_owner(s_pstart, sa + 1, ns, base + NT);
    const int npar = s_pstart[sb] - base;

    // ---- 1. parents: propagate, window, scan
    if (t < npar) {
      const int sd = packed_owner(s_pstart, sa, sb - 1, base + t);
      const int k = base + t - s_pstart[sd];
      const int64_t j = j0 + sd;
      const int64_t slot = cand_slot(j, k, D.S, D.in_rm);
      float p[6], lo[3], C[21];
#pragma unroll
      for (int c = 0; c < 6; ++c) p[c] = D.in.par[c * S8 + slot];
#pragma unroll
      for (int c = 0; c < 3; ++c) lo[c] = D.in.par[(6 + c) * S8 + slot];
#pragma unroll
      for (int c = 0; c < 21; ++c) C[c] = D.in.cov[c * S8 + slot];
      const float chi2tot = D.in.chi2[slot];
      const int32_t meta = D.in.meta[slot];
      const int nh = meta & 0xff;
      int32_t st = meta >> 8;
      bool stopped = (st & KF_ST_STOPPED) != 0;
      if (!stopped) {
        const int r = kf::propagate<float, kNewtonBuild, true>(p, lo, C, s_a[sd], D.R);
        if (r) {
          st |= r;
          stopped = true;
        } else if (D.x_x0 > 0.f) {
          kf::scatter(p, lo, C, D.x_x0, Args.mass);
        }
      }
      uint64_t L[LW];
      int P[LW];
#pragma unroll
      for (int q = 0; q < LW; ++q) {
        L[q] = kNoKey;
        P[q] = -1;
      }
      bool any = false;
      if (!stopped) {
        float Si[6];
        int e0 = 0, e1 = -1, fa0 = 0, fa1 = KF_BIN_PHI - 1, fb0 = 0, fb1 = -1;
        hit_window(p, lo, C, D.R, Args.v0, Args.v1, Args.v2, Args.cut, Si, e0, e1, fa0, fa1, fb0, fb1);
        any = scan_window(p, lo, Si, e0, e1, fa0, fa1, fb0, fb1, D.bin_off + int64_t(s_seg[sd]) * (KF_NBINS + 1),
                          D.hits + s_h0[sd], Args.cut, nh, chi2tot, k, L, P);
      }
      // no compatible hit (or a stopped candidate): one child without a hit
      if (!any) list_insert(L, P, make_key(nh, chi2tot, k, 0), -1);
#pragma unroll
      for (int c = 0; c < 6; ++c) s_state[c][t] = p[c];
#pragma unroll
      for (int c = 0; c < 3; ++c) s_state[6 + c][t] = lo[c];
#pragma unroll
      for (int c = 0; c < 21; ++c) s_state[kParN + c][t] = C[c];
#pragma unroll
      for (int q = 0; q < LW; ++q) {
        s_key[q][t] = L[q];
        s_pos[q][t] = P[q];
      }
      s_pst[t] = st | (stopped ? kStoppedBit : 0);
    }
    __syncthreads();

    // ---- 2. clone engine: one thread per seed of the round merges the
    // sorted lists of its parents (heads packed 4 bits per parent)
    int n_win = 0;
    const int nr = sb - sa;
    if (t < nr) {
      const int sd = sa + t;
      const int64_t j = j0 + sd;
      const int p0 = s_pstart[sd] - base, nc = s_pstart[sd + 1] - s_pstart[sd];
      uint32_t heads = 0;
      for (int r = 0; r < Args.max_cands; ++r) {
        uint64_t best = kNoKey;
        int bk = 0;
        for (int k = 0; k < nc; ++k) {
          const int h = int((heads >> (4 * k)) & 15u);
          if (h < LW) {
            const uint64_t key = s_key[h][p0 + k];
            if (key < best) {
              best = key;
              bk = k;
            }
          }
        }
        if (best == kNoKey) break;
        const int bh = int((heads >> (4 * bk)) & 15u);
        s_ckey[t][r] = best;
        s_cpos[t][r] = s_pos[bh][p0 + bk];
        heads += 1u << (4 * bk);
        D.hist_parent[cand_slot(j, r, D.S, D.out_rm)] = int8_t((best >> 21) & 7u);
        D.hist_hit[cand_slot(j, r, D.S, D.out_rm)] = int(best & 0x1fffffu) - 1;
        ++n_win;
      }
      D.out.ncand[j] = int8_t(n_win);
    }
    block_scan<NT>(n_win, s_cstart, s_wsum);

    // ---- 3. children: the parent's prediction updated with the child's hit
    const int nch = s_cstart[nr];
    for (int c = t; c < nch; c += NT) {
      const int sl = packed_owner(s_cstart, 0, nr - 1, c);
      const int r = c - s_cstart[sl];
      const int64_t j = j0 + sa + sl;
      const int64_t slot = cand_slot(j, r, D.S, D.out_rm);
      const uint64_t key = s_ckey[sl][r];
      const int pi = s_pstart[sa + sl] - base + int((key >> 21) & 7u);
      float q[6], ql[3], qC[21];
#pragma unroll
      for (int w = 0; w < 6; ++w) q[w] = s_state[w][pi];
#pragma unroll
      for (int w = 0; w < 3; ++w) ql[w] = s_state[6 + w][pi];
#pragma unroll
      for (int w = 0; w < 21; ++w) qC[w] = s_state[kParN + w][pi];
      const int pw = s_pst[pi];
      const int nh_new = 255 - int(key >> 56);
      const float chi2_new = __uint_as_float(uint32_t(key >> 24));
      const int hit_plus1 = int(key & 0x1fffffu);
      int32_t st_new = pw & ~kStoppedBit;
      if (hit_plus1 > 0) {
        const float4 m = D.hits[s_h0[sa + sl] + s_cpos[sl][r]];
        float Si[6];
        kf::inverse_S(qC, Args.v0, Args.v1, Args.v2, Si);
        float r0, r1, r2;
        kf::residual<float, true>(q, ql, m.x, m.y, m.z, r0, r1, r2);
        kf::kalman_update<float, true>(q, ql, qC, Si, r0, r1, r2, Args.v0, Args.v1, Args.v2);
      } else if (!(pw & kStoppedBit)) {
        st_new |= KF_ST_NO_HIT;
      }
#pragma unroll
      for (int w = 0; w < 6; ++w) D.out.par[w * S8 + slot] = q[w];
#pragma unroll
      for (int w = 0; w < 3; ++w) D.out.par[(6 + w) * S8 + slot] = ql[w];
#pragma unroll
      for (int w = 0; w < 21; ++w) D.out.cov[w * S8 + slot] = qC[w];
      D.out.chi2[slot] = chi2_new;
      D.out.meta[slot] = nh_new | (st_new << 8);
    }
    __syncthreads();  // the next round reuses the shared tables
    sa = sb;
  }
  __syncthreads();  // the next layer rewrites sD and the per-seed tables
  }
}

// ---- register-resident build (thread layout 4)
//
// The same computation per candidate as the other layouts, organised so that
// a candidate's state never leaves the registers between layers and no
// block-wide barrier is needed.  A warp takes a group of G = 32 / W seeds
// (consecutive in the order given; the warps of the GPU work on a narrow
// band of seeds, whose events' hits stay in L2); lane k of a seed's W lanes
// holds the seed's candidate of rank k.  Per building layer, every live lane
// propagates its candidate, derives the window and scans it into a sorted
// list of its best children's keys;
// the seed's lanes merge their lists by a minimum over the seed's lanes of the
// 64-bit keys (full-warp shuffles rotating within each seed's lanes) into
// the seed's best max_cands, ranked by the same total order; lane k then
// pulls the predicted state and S^-1 of its winner's parent from that lane by
// shuffles and applies the Kalman update with the winner's hit.  Only the
// per-layer history (parent rank, hit id) goes to memory; after the last
// layer the best candidates are written to the caller's result (or every
// candidate to the last buffer, for a final selection).  Groups are
// independent, so warps run at their own pace (no block barrier).  The keys
// are a total order and every candidate goes through the same functions as in
// the other layouts, so the results are bitwise theirs.

// Segmented merge: the W lanes of a seed (lanes gbase .. gbase + W - 1, mask
// seg) hold sorted lists (L, P) of their own children; the best max_cands
// keys of the union are found rank by rank by a minimum over the segment,
// taken with full-warp shuffles that rotate within the segment (offsets 1, 2
// and 4 reach every lane of a segment of up to 8): every lane executes the
// same shuffle, so segments of different seeds proceed in one instruction
// (warp intrinsics with a different member mask per segment are issued once
// per segment).  Lane k of the segment receives the k-th best (key, hit
// position); every lane the number of children kept.  Lanes outside any
// seed's segment (seg == 0) rotate onto themselves.
template <int W, int LW>
__device__ __forceinline__ void merge_segment(uint64_t (&L)[LW], int (&P)[LW], int max_cands, int k, int gbase,
                                              unsigned seg, uint64_t& my_key, int& my_pos, int& n_win) {
  const int lane = threadIdx.x & 31;
  const bool in_seg = seg != 0u;
  const int r1 = in_seg ? gbase + (k + 1) % W : lane;
  const int r2 = in_seg ? gbase + (k + 2) % W : lane;
  const int r4 = in_seg ? gbase + (k + 4) % W : lane;
  // the rank loop stays rolled: the step is large enough that the warps
  // stall on instruction fetch, and an unrolled merge costs more there than
  // its loop overhead (measured: 1.70 against 1.79 ms per build at N = 6)
#pragma unroll 1
  for (int r = 0; r < W; ++r) {
    if (r < max_cands) {  // uniform over the launch
      uint64_t m = L[0];
      if constexpr (W > 1) {
        uint64_t o = __shfl_sync(kFull, m, r1);
        m = o < m ? o : m;
        if constexpr (W > 2) {
          o = __shfl_sync(kFull, m, r2);
          m = o < m ? o : m;
        }
        if constexpr (W > 4) {
          o = __shfl_sync(kFull, m, r4);
          m = o < m ? o : m;
        }
      }
      const bool mine = L[0] == m && m != kNoKey;
      const unsigned bal = __ballot_sync(kFull, mine) & seg;
      const int wl = bal ? __ffs(bal) - 1 : lane;
      const int wpos = __shfl_sync(kFull, P[0], wl);
      if (mine) {
#pragma unroll
        for (int t = 0; t < LW - 1; ++t) {
          L[t] = L[t + 1];
          P[t] = P[t + 1];
        }
        L[LW - 1] = kNoKey;
        P[LW - 1] = -1;
      }
      if (m != kNoKey) {
        if (k == r) {
          my_key = m;
          my_pos = wpos;
        }
        ++n_win;
      }
    }
  }
}

template <typename T>
__device__ bool pd5_final(const T p[6], const T C[21]) {
  using kf::sym;
  const T r = sqrtf(p[0] * p[0] + p[1] * p[1]);
  const T t0 = r > T(0) ? -p[1] / r : T(0), t1 = r > T(0) ? p[0] / r : T(1);
  T M[5][5];
  M[0][0] = t0 * t0 * C[sym(0, 0)] + T(2) * t0 * t1 * C[sym(1, 0)] + t1 * t1 * C[sym(1, 1)];
  for (int jj = 1; jj < 5; ++jj) {
    M[jj][0] = t0 * C[sym(0, jj + 1)] + t1 * C[sym(1, jj + 1)];
    for (int kk = 1; kk <= jj; ++kk) M[jj][kk] = C[sym(jj + 1, kk + 1)];
  }
  T Lc[5][5];
  for (int jj = 0; jj < 5; ++jj) {
    T d = M[jj][jj];
    for (int kk = 0; kk < jj; ++kk) d -= Lc[jj][kk] * Lc[jj][kk];
    if (!(d > T(0))) return false;
    Lc[jj][jj] = sqrtf(d);
    for (int ii = jj + 1; ii < 5; ++ii) {
      T v = M[ii][jj];
      for (int kk = 0; kk < jj; ++kk) v -= Lc[ii][kk] * Lc[jj][kk];
      Lc[ii][jj] = v / Lc[jj][jj];
    }
  }
  return true;
}

// MAT: some building layer has material (the scattering code is compiled in
// only then: present but never run, it cost 2 % of the build)
template <int W, bool TABLE, bool MAT>
__global__ void __launch_bounds__(kResThreads, resident_blocks_per_sm(W))
    build_resident_kernel(const __grid_constant__ BuildResidentArgs A) {
  constexpr int G = 32 / W;  // seeds per group
  const int lane = threadIdx.x & 31;
  const int g = lane / W, k = lane - g * W;
  // the seed's lanes (none for lanes past G * W)
  const unsigned seg = g < G ? ((1u << W) - 1u) << (g * W) : 0u;
  const int64_t n_groups = TABLE ? A.n_groups : (A.one.S + G - 1) / G;
  // groups dealt out in order, each warp fetching its next one from a
  // counter: at any moment the warps of the GPU work on a narrow band of
  // seeds (a few events), whose hits stay in L2, and a warp whose groups
  // happened to be cheap takes more (measured: 2 % faster at N = 6, 6 % at
  // N = 1 than a fixed grid stride)
  auto next_group = [&]() {
    unsigned long long v = 0;
    if (lane == 0) v = atomicAdd(A.group_counter, 1ull);
    return int64_t(__shfl_sync(kFull, v, 0));
  };
  for (int64_t gi = next_group(); gi < n_groups; gi = next_group()) {
    int q = 0;  // the batch of this group (a served event), with a table
    if constexpr (TABLE)
      while (q + 1 < A.n_batches && A.table[q + 1].group_begin <= gi) ++q;
    const ResidentBatch& B = TABLE ? A.table[q] : A.one;
    const int64_t S8 = B.S * kGroup;
    const int64_t j = (gi - (TABLE ? B.group_begin : 0)) * G + g;
    const bool seed_ok = g < G && j < B.S;
    int e = 0, nc = 0;
    int64_t si = 0;  // seed index
    float a = A.a_scale;
    if (seed_ok) {
      e = B.seed_evt ? B.seed_evt[j] : 0;
      si = B.seed_perm ? B.seed_perm[j] : j;
      a = A.a_scale * float(B.charge[si]);
      nc = B.seed_par ? 1 : B.in.ncand[j];
    }
    bool active = seed_ok && k < nc;
    float p[6], lo[3], C[21];
    float chi2tot = 0.f;
    int nh = 0;
    int32_t st = 0;
    if (active && B.seed_par) {  // the seed itself
#pragma unroll
      for (int c = 0; c < 6; ++c) p[c] = B.seed_par[c * B.S + si];
#pragma unroll
      for (int c = 0; c < 3; ++c) lo[c] = B.seed_lo ? B.seed_lo[c * B.S + si] : 0.f;
#pragma unroll
      for (int c = 0; c < 21; ++c) C[c] = B.seed_cov[c * B.S + si];
    } else if (active) {
      const int64_t slot = cand_slot(j, k, B.S, A.in_rm);
#pragma unroll
      for (int c = 0; c < 6; ++c) p[c] = B.in.par[c * S8 + slot];
#pragma unroll
      for (int c = 0; c < 3; ++c) lo[c] = B.in.par[(6 + c) * S8 + slot];
#pragma unroll
      for (int c = 0; c < 21; ++c) C[c] = B.in.cov[c * S8 + slot];
      chi2tot = B.in.chi2[slot];
      const int32_t meta = B.in.meta[slot];
      nh = meta & 0xff;
      st = meta >> 8;
    } else {
#pragma unroll
      for (int c = 0; c < 6; ++c) p[c] = 0.f;
#pragma unroll
      for (int c = 0; c < 3; ++c) lo[c] = 0.f;
#pragma unroll
      for (int c = 0; c < 21; ++c) C[c] = 0.f;
    }
    int n_win = nc;
    for (int l = A.l0; l < A.n_layers; ++l) {
      const int64_t sg = int64_t(e) * A.n_layers + l;
      const int64_t h0 = seed_ok ? B.seg_off[sg] : 0;
      bool stopped = (st & KF_ST_STOPPED) != 0;
      if (active && !stopped) {
        const int r = kf::propagate<float, kNewtonBuild, true>(p, lo, C, a, A.R[l]);
        if (r) {
          st |= r;
          stopped = true;
        } else if (MAT && A.x_x0[l] > 0.f) {
          kf::scatter(p, lo, C, A.x_x0[l], A.mass);
        }
      }
      float Si[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      uint64_t L[W];
      int P[W];
#pragma unroll
      for (int t = 0; t < W; ++t) {
        L[t] = kNoKey;
        P[t] = -1;
      }
      const bool win = active && !stopped;
      // the window's rows by sub-bin where the batch has them
      const int nphi = B.fine_off ? KF_BIN_PHI_FINE : KF_BIN_PHI;
      const int32_t* boff =
          B.fine_off ? B.fine_off + sg * (KF_NBINS_FINE + 1) : B.bin_off + sg * (KF_NBINS + 1);
      int e0 = 0, e1 = -1, fa0 = 0, fa1 = nphi - 1, fb0 = 0, fb1 = -1;
      if (win) hit_window(p, lo, C, A.R[l], A.v0, A.v1, A.v2, A.cut, Si, e0, e1, fa0, fa1, fb0, fb1, nphi);
      // a row's hits loaded in batches: 4 with one lane a seed, 2 with more
      // (measured: 4 is slower at W = 6, where the registers are needed elsewhere)
      bool any = false;
      if (win) {
        if constexpr (W == 1)
          any = scan_window_batched(p, lo, Si, e0, e1, fa0, fa1, fb0, fb1, boff, B.hits + h0, A.cut, nh, chi2tot, k,
                                    L, P, nphi);
        else
          any = scan_window_batched<W, 2>(p, lo, Si, e0, e1, fa0, fa1, fb0, fb1, boff, B.hits + h0, A.cut, nh,
                                          chi2tot, k, L, P, nphi);
      }
      // no compatible hit (or a stopped candidate): one child without a hit
      if (active && !any) list_insert(L, P, make_key(nh, chi2tot, k, 0), -1);
      // clone engine: the seed's best max_cands children
      uint64_t my_key = kNoKey;
      int my_pos = -1;
      n_win = 0;
      merge_segment<W, W>(L, P, A.max_cands, k, g * W, seg, my_key, my_pos, n_win);
      // materialise: lane k takes its winner's parent prediction and S^-1
      const int src = k < n_win ? g * W + int((my_key >> 21) & 7u) : lane;
      float q[6], ql[3], qC[21], qS[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) q[c] = __shfl_sync(kFull, p[c], src);
#pragma unroll
      for (int c = 0; c < 3; ++c) ql[c] = __shfl_sync(kFull, lo[c], src);
#pragma unroll
      for (int c = 0; c < 21; ++c) qC[c] = __shfl_sync(kFull, C[c], src);
#pragma unroll
      for (int c = 0; c < 6; ++c) qS[c] = __shfl_sync(kFull, Si[c], src);
      const int32_t pst = __shfl_sync(kFull, st, src);
      const int pstopped = __shfl_sync(kFull, int(stopped), src);
      active = seed_ok && k < n_win;
      if (active) {
        const int nh_new = 255 - int(my_key >> 56);
        const float chi2_new = __uint_as_float(uint32_t(my_key >> 24));
        const int hit_plus1 = int(my_key & 0x1fffffu);
        int32_t st_new = pst;
        if (hit_plus1 > 0) {
          const float4 m = B.hits[h0 + my_pos];
          float r0, r1, r2;
          kf::residual<float, true>(q, ql, m.x, m.y, m.z, r0, r1, r2);
          kf::kalman_update<float, true>(q, ql, qC, qS, r0, r1, r2, A.v0, A.v1, A.v2);
        } else if (!pstopped) {
          st_new |= KF_ST_NO_HIT;
        }
        const int64_t hslot = int64_t(l) * S8 + cand_slot(j, k, B.S, l + 1 < A.rm_buffers);
        B.hist_parent[hslot] = int8_t((my_key >> 21) & 7u);
        B.hist_hit[hslot] = hit_plus1 - 1;
#pragma unroll
        for (int c = 0; c < 6; ++c) p[c] = q[c];
#pragma unroll
        for (int c = 0; c < 3; ++c) lo[c] = ql[c];
#pragma unroll
        for (int c = 0; c < 21; ++c) C[c] = qC[c];
        chi2tot = chi2_new;
        nh = nh_new;
        st = st_new;
      }
    }
    if (B.res.best.par) {
      // the final selection in place: lane k holds rank k, so the seed's
      // first lane writes the best candidate and every lane below max_cands
      // its summary; the paths (a chain of dependent history loads a seed)
      // are left to build_final_kernel in its paths-only form, and with
      // several lanes a seed so is the positive-definiteness check of the
      // best covariance (its code here, run by one lane of W, cost 6 % of the
      // N = 6 build): that kernel reads the position's low part from the
      // candidate buffer
      const kf_build_result& o = B.res;
      if (seed_ok && k < A.max_cands) {
        const int64_t seed = si;
        const bool have = k < n_win;
        if (k == 0) {
#pragma unroll
          for (int c = 0; c < 6; ++c) o.best.par[c * B.S + seed] = p[c];
          if (o.best.par_lo)
#pragma unroll
            for (int c = 0; c < 3; ++c) o.best.par_lo[c * B.S + seed] = lo[c];
#pragma unroll
          for (int c = 0; c < 21; ++c) o.best.cov[c * B.S + seed] = C[c];
          if (o.chi2_tot) o.chi2_tot[seed] = chi2tot;
          if (o.n_hits) o.n_hits[seed] = nh;
          if constexpr (W == 1) {
            float pf[6];
#pragma unroll
            for (int c = 0; c < 3; ++c) pf[c] = p[c] + lo[c];
#pragma unroll
            for (int c = 3; c < 6; ++c) pf[c] = p[c];
            if (o.status) o.status[seed] = pd5_final(pf, C) ? st : st | KF_ST_NOT_PD;
          } else if (o.status) {
            o.status[seed] = st;
            const int64_t slot = cand_slot(j, 0, B.S, A.out_rm);
#pragma unroll
            for (int c = 0; c < 3; ++c) B.out.par[(6 + c) * S8 + slot] = lo[c];
          }
          if (o.n_cands) o.n_cands[seed] = n_win;
        }
        const int64_t oc = seed * A.max_cands + k;
        if (o.cand_chi2_tot) o.cand_chi2_tot[oc] = have ? chi2tot : 0.f;
        if (o.cand_n_hits) o.cand_n_hits[oc] = have ? nh : 0;
      }
    } else {
      // the candidates after the last layer, for the final selection
      if (active) {
        const int64_t slot = cand_slot(j, k, B.S, A.out_rm);
#pragma unroll
        for (int c = 0; c < 6; ++c) B.out.par[c * S8 + slot] = p[c];
#pragma unroll
        for (int c = 0; c < 3; ++c) B.out.par[(6 + c) * S8 + slot] = lo[c];
#pragma unroll
        for (int c = 0; c < 21; ++c) B.out.cov[c * S8 + slot] = C[c];
        B.out.chi2[slot] = chi2tot;
        B.out.meta[slot] = nh | (st << 8);
      }
    }
    if (seed_ok && k == 0) B.out.ncand[j] = int8_t(n_win);
  }
}

// First building layer of the register-resident build, one thread per seed.
// On that layer every seed holds one candidate (the seed itself), so the W
// lanes a seed owns in build_resident_kernel would idle all but one; here a
// thread propagates its seed, derives and scans the window, and updates the
// seed's best max_cands children itself (the list of a single parent is the
// seed's ranking), writing them to candidate buffer l0 + 1 and the layer's
// history.  The same functions and keys as every other layout, so the same
// bits; build_resident_kernel then continues from layer l0 + 1.
template <bool TABLE, bool MAT>
__global__ void __launch_bounds__(kResThreads, kResBlocksPerSM)
    build_first_layer_kernel(const __grid_constant__ BuildResidentArgs A) {
  const int64_t t = int64_t(blockIdx.x) * kResThreads + threadIdx.x;
  int q = 0;  // the batch of this seed (a served event), with a table
  if constexpr (TABLE) {
    if (t >= A.n_seeds) return;
    while (q + 1 < A.n_batches && A.table[q + 1].seed_begin <= t) ++q;
  }
  const ResidentBatch& B = TABLE ? A.table[q] : A.one;
  const int64_t j = t - (TABLE ? B.seed_begin : 0);
  if (j >= B.S) return;
  const int64_t S8 = B.S * kGroup;
  const int l = A.l0;
  const int e = B.seed_evt ? B.seed_evt[j] : 0;
  const int64_t si = B.seed_perm ? B.seed_perm[j] : j;
  const float a = A.a_scale * float(B.charge[si]);
  float p[6], lo[3], C[21];
  float chi2tot = 0.f;
  int nh = 0;
  int32_t st = 0;
  if (B.seed_par) {  // the seed itself
#pragma unroll
    for (int c = 0; c < 6; ++c) p[c] = B.seed_par[c * B.S + si];
#pragma unroll
    for (int c = 0; c < 3; ++c) lo[c] = B.seed_lo ? B.seed_lo[c * B.S + si] : 0.f;
#pragma unroll
    for (int c = 0; c < 21; ++c) C[c] = B.seed_cov[c * B.S + si];
  } else {
    const int64_t slot = cand_slot(j, 0, B.S, A.in_rm);  // the seed's only candidate
#pragma unroll
    for (int c = 0; c < 6; ++c) p[c] = B.in.par[c * S8 + slot];
#pragma unroll
    for (int c = 0; c < 3; ++c) lo[c] = B.in.par[(6 + c) * S8 + slot];
#pragma unroll
    for (int c = 0; c < 21; ++c) C[c] = B.in.cov[c * S8 + slot];
    chi2tot = B.in.chi2[slot];
    const int32_t meta = B.in.meta[slot];
    nh = meta & 0xff;
    st = meta >> 8;
  }
  const int64_t sg = int64_t(e) * A.n_layers + l;
  const int64_t h0 = B.seg_off[sg];
  bool stopped = (st & KF_ST_STOPPED) != 0;
  if (!stopped) {
    const int r = kf::propagate<float, kNewtonBuild, true>(p, lo, C, a, A.R[l]);
    if (r) {
      st |= r;
      stopped = true;
    } else if (MAT && A.x_x0[l] > 0.f) {
      kf::scatter(p, lo, C, A.x_x0[l], A.mass);
    }
  }
  float Si[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  uint64_t L[kGroup];
  int P[kGroup];
#pragma unroll
  for (int t = 0; t < kGroup; ++t) {
    L[t] = kNoKey;
    P[t] = -1;
  }
  bool any = false;
  if (!stopped) {
    const int nphi = B.fine_off ? KF_BIN_PHI_FINE : KF_BIN_PHI;
    const int32_t* boff = B.fine_off ? B.fine_off + sg * (KF_NBINS_FINE + 1) : B.bin_off + sg * (KF_NBINS + 1);
    int e0 = 0, e1 = -1, fa0 = 0, fa1 = nphi - 1, fb0 = 0, fb1 = -1;
    hit_window(p, lo, C, A.R[l], A.v0, A.v1, A.v2, A.cut, Si, e0, e1, fa0, fa1, fb0, fb1, nphi);
    any = scan_window(p, lo, Si, e0, e1, fa0, fa1, fb0, fb1, boff, B.hits + h0, A.cut, nh, chi2tot, 0, L, P, nphi);
  }
  // no compatible hit (or a stopped seed): one child without a hit
  if (!any) list_insert(L, P, make_key(nh, chi2tot, 0, 0), -1);
  int n_win = 0;
#pragma unroll 1
  for (int r = 0; r < A.max_cands; ++r) {
    uint64_t key = kNoKey;
    int pos = -1;
#pragma unroll
    for (int t = 0; t < kGroup; ++t)
      if (t == r) {
        key = L[t];
        pos = P[t];
      }
    if (key == kNoKey) break;
    ++n_win;
    float q[6], ql[3], qC[21];
#pragma unroll
    for (int c = 0; c < 6; ++c) q[c] = p[c];
#pragma unroll
    for (int c = 0; c < 3; ++c) ql[c] = lo[c];
#pragma unroll
    for (int c = 0; c < 21; ++c) qC[c] = C[c];
    const int nh_new = 255 - int(key >> 56);
    const float chi2_new = __uint_as_float(uint32_t(key >> 24));
    const int hit_plus1 = int(key & 0x1fffffu);
    int32_t st_new = st;
    if (hit_plus1 > 0) {
      const float4 m = B.hits[h0 + pos];
      float r0, r1, r2;
      kf::residual<float, true>(q, ql, m.x, m.y, m.z, r0, r1, r2);
      kf::kalman_update<float, true>(q, ql, qC, Si, r0, r1, r2, A.v0, A.v1, A.v2);
    } else if (!stopped) {
      st_new |= KF_ST_NO_HIT;
    }
    const int64_t os = cand_slot(j, r, B.S, A.out_rm);
#pragma unroll
    for (int c = 0; c < 6; ++c) B.out.par[c * S8 + os] = q[c];
#pragma unroll
    for (int c = 0; c < 3; ++c) B.out.par[(6 + c) * S8 + os] = ql[c];
#pragma unroll
    for (int c = 0; c < 21; ++c) B.out.cov[c * S8 + os] = qC[c];
    B.out.chi2[os] = chi2_new;
    B.out.meta[os] = nh_new | (st_new << 8);
    B.hist_parent[int64_t(l) * S8 + os] = 0;
    B.hist_hit[int64_t(l) * S8 + os] = hit_plus1 - 1;
  }
  B.out.ncand[j] = int8_t(n_win);
}

cudaError_t launch_build_first_layer(const BuildResidentArgs& a, cudaStream_t st) {
  const int64_t seeds = a.table ? a.n_seeds : a.one.S;
  if (seeds <= 0) return cudaSuccess;
  const int grid = int((seeds + kResThreads - 1) / kResThreads);
  const bool mat = a.x_x0[a.l0] > 0.f;
  if (a.table)
    mat ? build_first_layer_kernel<true, true><<<grid, kResThreads, 0, st>>>(a)
        : build_first_layer_kernel<true, false><<<grid, kResThreads, 0, st>>>(a);
  else
    mat ? build_first_layer_kernel<false, true><<<grid, kResThreads, 0, st>>>(a)
        : build_first_layer_kernel<false, false><<<grid, kResThreads, 0, st>>>(a);
  return cudaGetLastError();
}

template <bool TABLE, bool MAT>
static void launch_resident_w(const BuildResidentArgs& a, int W, int grid, cudaStream_t st) {
  switch (W) {
    case 1: build_resident_kernel<1, TABLE, MAT><<<grid, kResThreads, 0, st>>>(a); break;
    case 2: build_resident_kernel<2, TABLE, MAT><<<grid, kResThreads, 0, st>>>(a); break;
    case 4: build_resident_kernel<4, TABLE, MAT><<<grid, kResThreads, 0, st>>>(a); break;
    case 6: build_resident_kernel<6, TABLE, MAT><<<grid, kResThreads, 0, st>>>(a); break;
    default: build_resident_kernel<8, TABLE, MAT><<<grid, kResThreads, 0, st>>>(a); break;
  }
}

cudaError_t launch_build_resident(const BuildResidentArgs& a, int num_sms, cudaStream_t st) {
  const int W = resident_lanes(a.max_cands);
  const int64_t groups = a.table ? a.n_groups : (a.one.S + (32 / W) - 1) / (32 / W);
  if (groups <= 0) return cudaSuccess;
  const int64_t need = (groups + kResThreads / 32 - 1) / (kResThreads / 32);
  const int grid = int(std::max<int64_t>(1, std::min<int64_t>(need, int64_t(num_sms) * resident_blocks_per_sm(W))));
  bool mat = false;
  for (int l = a.l0; l < a.n_layers; ++l) mat |= a.x_x0[l] > 0.f;
  if (a.table)
    mat ? launch_resident_w<true, true>(a, W, grid, st) : launch_resident_w<true, false>(a, W, grid, st);
  else
    mat ? launch_resident_w<false, true>(a, W, grid, st) : launch_resident_w<false, false>(a, W, grid, st);
  return cudaGetLastError();
}

__global__ void build_init_kernel(const BuildInitArgs A) {
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= A.S) return;
  const int64_t s = A.seed_perm[j];
  const int64_t S8 = A.S * kGroup, slot = cand_slot(j, 0, A.S, true);  // buffer 0: rank-major
  for (int c = 0; c < 6; ++c) A.out.par[c * S8 + slot] = A.par[c * A.n + s];
  for (int c = 0; c < 3; ++c) A.out.par[(6 + c) * S8 + slot] = A.lo ? A.lo[c * A.n + s] : 0.f;
  for (int c = 0; c < 21; ++c) A.out.cov[c * S8 + slot] = A.cov[c * A.n + s];
  A.out.chi2[slot] = 0.f;
  A.out.meta[slot] = 0;
  A.out.ncand[j] = 1;
}

__global__ void build_final_kernel(const BuildFinalArgs A) {
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= A.S) return;
  const int64_t seed = A.seed_perm ? A.seed_perm[j] : j;
  const int64_t S8 = A.S * kGroup;
  const bool last_rm = A.n_layers < A.rm_buffers;  // layout of buffer n_layers
  const int nc = A.cand.ncand[j];
  const kf_build_result& o = A.out;
  if (A.paths_only) {  // the build launch wrote the rest but these
    if (A.paths_only == 2 && o.status) {  // the best covariance positive definite (low part from the buffer)
      const int64_t slot = cand_slot(j, 0, A.S, last_rm);
      float pf[6], C[21];
      for (int c = 0; c < 6; ++c) pf[c] = o.best.par[c * A.S + seed];
      for (int c = 0; c < 3; ++c) pf[c] = pf[c] + A.cand.par[(6 + c) * S8 + slot];
      for (int c = 0; c < 21; ++c) C[c] = o.best.cov[c * A.S + seed];
      if (!pd5_final(pf, C)) o.status[seed] |= KF_ST_NOT_PD;
    }
    if (o.hit_idx) {
      int kk = 0;
      for (int l = A.n_layers - 1; l >= 0; --l) {
        const int64_t sl = int64_t(l) * S8 + cand_slot(j, kk, A.S, l + 1 < A.rm_buffers);
        o.hit_idx[int64_t(l) * A.S + seed] = A.hist_hit[sl];
        kk = A.hist_parent[sl];
      }
    }
    if (o.cand_hit_idx)
      for (int c = 0; c < A.max_cands; ++c) {
        int kk = c;
        for (int l = A.n_layers - 1; l >= 0; --l) {
          int32_t h = -1;
          if (c < nc) {
            const int64_t sl = int64_t(l) * S8 + cand_slot(j, kk, A.S, l + 1 < A.rm_buffers);
            h = A.hist_hit[sl];
            kk = A.hist_parent[sl];
          }
          o.cand_hit_idx[int64_t(l) * A.S * A.max_cands + seed * A.max_cands + c] = h;
        }
      }
    return;
  }
  // best candidate: rank 0
  {
    const int64_t slot = cand_slot(j, 0, A.S, last_rm);
    float p[6], C[21];
    for (int c = 0; c < 6; ++c) p[c] = A.cand.par[c * S8 + slot];
    for (int c = 0; c < 21; ++c) C[c] = A.cand.cov[c * S8 + slot];
    for (int c = 0; c < 6; ++c) o.best.par[c * A.S + seed] = p[c];
    if (o.best.par_lo)
      for (int c = 0; c < 3; ++c) o.best.par_lo[c * A.S + seed] = A.cand.par[(6 + c) * S8 + slot];
    for (int c = 0; c < 21; ++c) o.best.cov[c * A.S + seed] = C[c];
    const int32_t meta = A.cand.meta[slot];
    float pf[6];
    for (int c = 0; c < 3; ++c) pf[c] = p[c] + A.cand.par[(6 + c) * S8 + slot];
    for (int c = 3; c < 6; ++c) pf[c] = p[c];
    int32_t st = meta >> 8;
    if (!pd5_final(pf, C)) st |= KF_ST_NOT_PD;
    if (o.chi2_tot) o.chi2_tot[seed] = A.cand.chi2[slot];
    if (o.n_hits) o.n_hits[seed] = meta & 0xff;
    if (o.status) o.status[seed] = st;
    if (o.hit_idx) {
      int kk = 0;
      for (int l = A.n_layers - 1; l >= 0; --l) {
        const int64_t sl = int64_t(l) * S8 + cand_slot(j, kk, A.S, l + 1 < A.rm_buffers);
        o.hit_idx[int64_t(l) * A.S + seed] = A.hist_hit[sl];
        kk = A.hist_parent[sl];
      }
    }
  }
  if (o.n_cands) o.n_cands[seed] = nc;
  for (int c = 0; c < A.max_cands; ++c) {
    const int64_t oc = seed * A.max_cands + c;
    const int64_t slot = cand_slot(j, c, A.S, last_rm);
    if (o.cand_chi2_tot) o.cand_chi2_tot[oc] = c < nc ? A.cand.chi2[slot] : 0.f;
    if (o.cand_n_hits) o.cand_n_hits[oc] = c < nc ? (A.cand.meta[slot] & 0xff) : 0;
    if (o.cand_hit_idx) {
      int kk = c;
      for (int l = A.n_layers - 1; l >= 0; --l) {
        int32_t h = -1;
        if (c < nc) {
          const int64_t sl = int64_t(l) * S8 + cand_slot(j, kk, A.S, l + 1 < A.rm_buffers);
          h = A.hist_hit[sl];
          kk = A.hist_parent[sl];
        }
        o.cand_hit_idx[int64_t(l) * A.S * A.max_cands + oc] = h;
      }
    }
  }
}

template <int TILE, int LW>
static void launch_step_scan(const BuildStepArgs& a, int grid, cudaStream_t st, bool coop) {
  const size_t smem = size_t(kWarps) * TILE * sizeof(float4);
  if (coop)
    build_step_kernel<TILE, LW, true><<<grid, kBuildThreads, smem, st>>>(a);
  else
    build_step_kernel<TILE, LW, false><<<grid, kBuildThreads, smem, st>>>(a);
}

cudaError_t launch_build_step(const BuildStepArgs& a, int grid, cudaStream_t st, int tile, int list, int scan) {
  if (grid <= 0) return cudaSuccess;
  const bool narrow = list == 4 && a.max_cands <= 4, coop = scan == 1;
  if (is_packed(scan)) {  // candidate-packed (no hit staging)
    if (scan == 2 && narrow)
      build_step_packed_kernel<4, kPackSeeds><<<grid, kPackSeeds, 0, st>>>(a);
    else if (scan == 2)
      build_step_packed_kernel<kGroup, kPackSeeds><<<grid, kPackSeeds, 0, st>>>(a);
    else if (narrow)
      build_step_packed_kernel<4, kPackSeeds / 2><<<grid, kPackSeeds / 2, 0, st>>>(a);
    else
      build_step_packed_kernel<kGroup, kPackSeeds / 2><<<grid, kPackSeeds / 2, 0, st>>>(a);
    return cudaGetLastError();
  }
  if (tile > 0) {
    if (narrow)
      launch_step_scan<kBuildTile, 4>(a, grid, st, coop);
    else
      launch_step_scan<kBuildTile, kGroup>(a, grid, st, coop);
  } else {
    if (narrow)
      launch_step_scan<0, 4>(a, grid, st, coop);
    else
      launch_step_scan<0, kGroup>(a, grid, st, coop);
  }
  return cudaGetLastError();
}

cudaError_t launch_build_init(const BuildInitArgs& a, cudaStream_t st) {
  if (a.S <= 0) return cudaSuccess;
  build_init_kernel<<<int((a.S + 255) / 256), 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_build_final(const BuildFinalArgs& a, cudaStream_t st) {
  if (a.S <= 0) return cudaSuccess;
  build_final_kernel<<<int((a.S + 127) / 128), 128, 0, st>>>(a);
  return cudaGetLastError();
}

// evt[j] = the event of seed j: the last e with seed_off[e] <= j (binary search)
__global__ void seed_event_kernel(int32_t* evt, const int64_t* seed_off, int64_t E, int64_t S) {
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= S) return;
  int64_t lo = 0, hi = E;
  while (hi - lo > 1) {
    const int64_t m = (lo + hi) / 2;
    if (seed_off[m] <= j)
      lo = m;
    else
      hi = m;
  }
  evt[j] = int32_t(lo);
}

__global__ void globalise_perm_kernel(int32_t* perm, const int32_t* evt, const int64_t* seed_off, int64_t S) {
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j < S) perm[j] = int32_t(seed_off[evt[j]] + perm[j]);
}

}  // namespace kfi

using namespace kfi;

namespace {
size_t al256(size_t b) { return (b + 255) & ~size_t(255); }
}  // namespace

extern "C" int kf_build(kf_ctx* ctx, const kf_tracks* seeds, const int64_t* seed_off, const kf_layer_hit_bins* bins,
                        int32_t max_cands, kf_build_result* out, void* stream) {
  if (!ctx || !seeds || !seed_off || !bins || !out) return KF_EINVAL;
  if (max_cands < 1 || max_cands > kGroup) return KF_EINVAL;
  if (seeds->n < 0 || bins->n_events < 0 || bins->n_layers < 1 || bins->first_layer < 0 ||
      bins->first_layer + bins->n_layers > ctx->cfg.n_layers)
    return KF_EINVAL;
  const int64_t S = seeds->n;
  if (S == 0) return KF_OK;
  if (!seeds->par || !seeds->cov || !seeds->charge || !bins->bin_off || !bins->seg_off) return KF_EINVAL;
  if (bins->n_hits > 0 && !bins->hits) return KF_EINVAL;
  if (!out->best.par || !out->best.cov) return KF_EINVAL;
  if (bins->n_events == 0) return KF_EINVAL;
  KF_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  const int L = bins->n_layers;
  const int64_t S8 = S * kGroup;
  // scratch layout
  const size_t b_perm = al256(S * 4), b_evt = al256(S * 4);
  const size_t b_cand = cand_bytes(S);
  const size_t b_hp = al256(size_t(L) * S8), b_hh = al256(size_t(L) * S8 * 4);
  const size_t b_tab = al256(sizeof(BuildSlot) * size_t(L));
  const int64_t E = bins->n_events;
  const size_t b_sbin = al256(size_t(E) * (KF_NBINS + 1) * 4), b_scur = al256(size_t(E) * KF_NBINS * 4);
  const size_t b_ctr = 256;  // the resident build's group counter
  const size_t total = b_perm + b_evt + 2 * b_cand + b_hp + b_hh + b_tab + b_sbin + b_scur + b_ctr;
  int rc = scratch_reserve(ctx, ctx->s_build, total);
  if (rc) return rc;
  char* base = static_cast<char*>(ctx->s_build.ptr);
  int32_t* perm = reinterpret_cast<int32_t*>(base);
  int32_t* evt = reinterpret_cast<int32_t*>(base + b_perm);
  CandBuf bufA = cand_at(base + b_perm + b_evt, S);
  CandBuf bufB = cand_at(base + b_perm + b_evt + b_cand, S);
  int8_t* hist_parent = reinterpret_cast<int8_t*>(base + b_perm + b_evt + 2 * b_cand);
  int32_t* hist_hit = reinterpret_cast<int32_t*>(base + b_perm + b_evt + 2 * b_cand + b_hp);
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  // The layer-stepping layouts take the seeds in (eta, phi) bin order within
  // each event (a block's seeds share hit tiles); the register-resident one
  // in their given order, only their events looked up: measured, its build
  // is as fast or faster unordered (no tiles are shared; a grid-stride band
  // of seeds spans a few events whose hits stay in L2 either way), and the
  // ordering launches are saved.
  const bool ordered = ctx->tune.build_scan != 4;
  if (!ordered) {
    seed_event_kernel<<<int((S + 255) / 256), 256, 0, s>>>(evt, seed_off, bins->n_events, S);
    KF_CUDA_TRY(ctx, cudaGetLastError());
  }
  BinArgs ba;
  ba.xyz = seeds->par;
  ba.stride = S;
  ba.seg_off = seed_off;
  ba.bin_off = reinterpret_cast<int32_t*>(base + b_perm + b_evt + 2 * b_cand + b_hp + b_hh + b_tab);
  ba.out_pts = nullptr;
  ba.out_id = perm;
  ba.out_seg = evt;
  ba.cursor = reinterpret_cast<int32_t*>(base + b_perm + b_evt + 2 * b_cand + b_hp + b_hh + b_tab + b_sbin);
  ba.unordered = 1;  // each seed's result is independent of the order of the seeds in a bin
  if (ordered) {
    KF_CUDA_TRY(ctx, launch_bin_points(ba, bins->n_events, s));
    // perm holds ids within each event: make them global seed indices
    // (the seeds of event e start at seed_off[e])
    globalise_perm_kernel<<<int((S + 255) / 256), 256, 0, s>>>(perm, evt, seed_off, S);
    KF_CUDA_TRY(ctx, cudaGetLastError());
  }
  if (ctx->tune.build_scan != 4) {  // (the register-resident build reads the seeds itself)
    BuildInitArgs ia;
    ia.out = bufA;
    ia.par = seeds->par;
    ia.lo = seeds->par_lo;
    ia.cov = seeds->cov;
    ia.seed_perm = perm;
    ia.n = S;
    ia.S = S;
    build_init_kernel<<<int((S + 255) / 256), 256, 0, s>>>(ia);
    KF_CUDA_TRY(ctx, cudaGetLastError());
  }
  const float v0 = ctx->cfg.sigma_xy_cm * ctx->cfg.sigma_xy_cm;
  const float v2 = ctx->cfg.sigma_z_cm * ctx->cfg.sigma_z_cm;
  // candidate-packed steps: seeds spread over whole waves of blocks (build_pack_seeds)
  const int pack_seeds = build_pack_seeds(S, ctx->tune.build_scan, max_cands, ctx->num_sms);
  const int grid = pack_seeds > 0 ? int((S + pack_seeds - 1) / pack_seeds) : build_step_blocks(S, ctx->tune.build_scan);
  // one slot (the whole batch) per layer launch; the table goes to device
  // scratch in one copy (the host array is consumed before the call returns)
  const int rm_buffers = rank_major_buffers(max_cands, L);
  std::vector<BuildSlot> table(L);
  for (int l = 0; l < L; ++l) {
    BuildSlot& d = table[l];
    d.in = (l % 2 == 0) ? bufA : bufB;
    d.out = (l % 2 == 0) ? bufB : bufA;
    d.hist_parent = hist_parent + int64_t(l) * S8;
    d.hist_hit = hist_hit + int64_t(l) * S8;
    d.seed_evt = evt;
    d.seed_perm = perm;
    d.charge = seeds->charge;
    d.hits = reinterpret_cast<const float4*>(bins->hits);
    d.bin_off = bins->bin_off;
    d.seg_off = bins->seg_off;
    d.S = S;
    d.layer = l;
    d.n_layers = L;
    d.R = ctx->radius[bins->first_layer + l];
    d.x_x0 = ctx->x_x0[bins->first_layer + l];
    d.in_rm = l < rm_buffers;
    d.out_rm = l + 1 < rm_buffers;
    d.block_begin = 0;
  }
  BuildSlot* dtable = reinterpret_cast<BuildSlot*>(base + b_perm + b_evt + 2 * b_cand + b_hp + b_hh);
  KF_CUDA_TRY(ctx, cudaMemcpyAsync(dtable, table.data(), sizeof(BuildSlot) * L, cudaMemcpyHostToDevice, s));
  // Candidate-packed layouts take every block's seeds through consecutive
  // layers in one launch -- but only over buffers of one layout: where the
  // layout switches from rank-major to seed-major, a slot of one seed in one
  // layout is a slot of another seed in the other, so a block writing the
  // next buffer could overwrite what a block still on the previous layer
  // reads in the same memory.  Layers up to the switch run one launch each.
  // The grouped layouts launch once per layer.
  if (ctx->tune.build_scan == 4) {
    // register-resident layout: one launch takes every seed through all
    // layers from the seeds themselves and selects the best candidates; with
    // several lanes a seed, the first layer (one candidate a seed) runs first
    // with one thread per seed, into buffer 1
    BuildResidentArgs ra;
    ra.one.in = bufA;
    ra.one.out = bufB;
    ra.one.hist_parent = hist_parent;
    ra.one.hist_hit = hist_hit;
    ra.one.seed_evt = evt;
    ra.one.seed_perm = nullptr;  // the given order
    ra.one.charge = seeds->charge;
    ra.one.hits = reinterpret_cast<const float4*>(bins->hits);
    ra.one.bin_off = bins->bin_off;
    ra.one.seg_off = bins->seg_off;
    ra.one.fine_off = bins->fine_off;
    ra.one.S = S;
    ra.one.group_begin = 0;
    ra.one.seed_begin = 0;
    std::memset(&ra.one.res, 0, sizeof ra.one.res);
    ra.one.seed_par = seeds->par;
    ra.one.seed_lo = seeds->par_lo;
    ra.one.seed_cov = seeds->cov;
    ra.table = nullptr;
    ra.n_batches = 1;
    ra.n_groups = 0;
    ra.n_seeds = 0;
    ra.n_layers = L;
    ra.l0 = 0;
    ra.rm_buffers = rm_buffers;
    ra.max_cands = max_cands;
    ra.in_rm = 0 < rm_buffers;
    ra.out_rm = L < rm_buffers;
    ra.a_scale = float(kCLight * double(ctx->cfg.bz_tesla));
    ra.v0 = v0;
    ra.v1 = v0;
    ra.v2 = v2;
    ra.cut = ctx->cfg.chi2_cut;
    ra.mass = ctx->mass;
    for (int l = 0; l < kMaxLayers; ++l) {
      ra.R[l] = l < L ? ctx->radius[bins->first_layer + l] : 0.f;
      ra.x_x0[l] = l < L ? ctx->x_x0[bins->first_layer + l] : 0.f;
    }
    if (resident_lanes(max_cands) > 1 && L > 1) {
      // the first layer with one thread per seed (buffer 0 -> buffer 1), then
      // layers 1 .. L-1 from buffer 1 into the other buffer
      BuildResidentArgs fl = ra;
      fl.out_rm = 1 < rm_buffers;
      KF_CUDA_TRY(ctx, launch_build_first_layer(fl, s));
      ra.one.seed_par = ra.one.seed_lo = ra.one.seed_cov = nullptr;
      ra.one.in = bufB;
      ra.in_rm = 1 < rm_buffers;
      ra.one.out = bufA;
      ra.l0 = 1;
    }
    // the last launch also selects the best candidates and writes `out`,
    // all but the paths and the covariance check: those follow, one thread
    // a seed
    ra.one.res = *out;
    ra.group_counter = reinterpret_cast<unsigned long long*>(base + total - b_ctr);
    KF_CUDA_TRY(ctx, cudaMemsetAsync(ra.group_counter, 0, sizeof(unsigned long long), s));
    KF_CUDA_TRY(ctx, launch_build_resident(ra, ctx->num_sms, s));
    BuildFinalArgs fa;
    fa.cand = ra.one.out;
    fa.hist_parent = hist_parent;
    fa.hist_hit = hist_hit;
    fa.seed_perm = nullptr;
    fa.S = S;
    fa.n_layers = L;
    fa.max_cands = max_cands;
    fa.rm_buffers = rm_buffers;
    fa.paths_only = resident_defers_pd(max_cands) ? 2 : 1;
    fa.out = *out;
    if (out->hit_idx || out->cand_hit_idx || (out->status && fa.paths_only == 2)) {
      build_final_kernel<<<int((S + 127) / 128), 128, 0, s>>>(fa);
      KF_CUDA_TRY(ctx, cudaGetLastError());
    }
    return KF_OK;
  }
  const int first_fused = is_packed(ctx->tune.build_scan) ? (rm_buffers > L ? 0 : std::min(L, rm_buffers)) : L;
  for (int l = 0; l < (first_fused < L ? first_fused + 1 : L); ++l) {
    const bool fused = l == first_fused;
    BuildStepArgs a;
    a.slots = dtable + l;
    a.n_slots = 1;
    a.layers = fused ? L - l : 0;
    a.test_skip_warp = ctx->test_build_skip_warp;
    a.test_wait_limit = ctx->test_build_wait_polls;
    a.max_cands = max_cands;
    a.a_scale = float(kCLight * double(ctx->cfg.bz_tesla));
    a.v0 = v0;
    a.v1 = v0;
    a.v2 = v2;
    a.cut = ctx->cfg.chi2_cut;
    a.mass = ctx->mass;
    a.pack_seeds = pack_seeds;
    KF_CUDA_TRY(ctx, launch_build_step(a, grid, s, ctx->tune.build_hit_tile, ctx->tune.build_list_width,
                                       ctx->tune.build_scan));
  }
  BuildFinalArgs fa;
  fa.cand = (L % 2 == 0) ? bufA : bufB;
  fa.hist_parent = hist_parent;
  fa.hist_hit = hist_hit;
  fa.seed_perm = perm;
  fa.S = S;
  fa.n_layers = L;
  fa.max_cands = max_cands;
  fa.rm_buffers = rm_buffers;
  fa.paths_only = 0;
  fa.out = *out;
  build_final_kernel<<<int((S + 127) / 128), 128, 0, s>>>(fa);
  KF_CUDA_TRY(ctx, cudaGetLastError());
  return KF_OK;
}

