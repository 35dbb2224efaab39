// kf_build_f64.cu -- the plain double-precision form of the combinatorial
// build (Cerati et al., Sec. 3): the comparison form of the batched FP32
// build, written the straightforward way.
//
// One thread per seed, one launch per event and building layer.  A thread
// takes each of its seed's candidates in turn: propagates it (the same
// templates as the FP32 kernels, in double, no position pair), derives the
// chi2 window in double, scans the window's bins (the binned hits of
// kf_bin_hits) and keeps the seed's best max_cands children in one sorted
// list ranked by (nHits desc, chi2_tot asc, parent rank asc, hit id asc); then
// it updates each kept child from its parent's prediction, held in the
// thread's local memory, and stores it.  Candidates live in global double
// buffers between the per-layer launches; no thread layout, packing, staging
// or register residency: the plain form against which the batched FP32 form's
// events/s factor is stated.
#include <algorithm>
#include <cmath>
#include <vector>

#include "kf_bin.cuh"
#include "kf_internal.h"
#include "kf_math.cuh"

namespace kfi {
namespace {

constexpr int kNewtonBuild64 = 16;
constexpr int kF64Threads = 128;
constexpr int kF64MaxCands = 8;

// Candidate buffer of the FP64 build: slot j * max_cands + k holds candidate
// k of seed j; components structure-of-arrays over the S * max_cands slots.
struct CandF64 {
  double* par;     // [6][SM]
  double* cov;     // [21][SM]
  double* chi2;    // [SM] chi2_tot
  int32_t* meta;   // [SM] nHits | status << 8
  int8_t* ncand;   // [S]
};

struct StepF64Args {
  CandF64 in, out;
  int8_t* hist_parent;  // [SM] of this layer
  int32_t* hist_hit;    // [SM] of this layer
  const int8_t* charge;
  const float4* hits;   // binned hits of the batch
  const int32_t* bin_off;
  const int64_t* seg_off;
  int64_t S, begin, end;  // seeds of this event: [begin, end)
  int seg;                // segment (event, layer)
  int max_cands;
  double a_scale, R, x_x0, mass, v0, v1, v2, cut;
};

struct Child {
  int nh;
  double chi2;
  int parent, hit, pos;  // hit id (-1: none) and its position in the binned hits
};

__device__ __forceinline__ bool child_before(const Child& a, const Child& b) {
  if (a.nh != b.nh) return a.nh > b.nh;
  if (a.chi2 != b.chi2) return a.chi2 < b.chi2;
  if (a.parent != b.parent) return a.parent < b.parent;
  return a.hit < b.hit;
}

__device__ __forceinline__ void keep_child(Child* list, int& n, int cap, const Child& c) {
  if (n == cap && !child_before(c, list[n - 1])) return;
  int i = n < cap ? n++ : n - 1;
  while (i > 0 && child_before(c, list[i - 1])) {
    list[i] = list[i - 1];
    --i;
  }
  list[i] = c;
}

__device__ __forceinline__ int eta_bin64(double eta) {
  const int b = int(floor((eta + double(KF_BIN_ETA_MAX)) * (double(KF_BIN_ETA) / (2.0 * double(KF_BIN_ETA_MAX)))));
  return b < 0 ? 0 : (b >= KF_BIN_ETA ? KF_BIN_ETA - 1 : b);
}

// The chi2 window in double: for any unit u, chi2 >= (u.r)^2 / (u^T S u), so
// a hit with chi2 < cut lies within wt, wn, wz of the prediction along the
// tangent, the normal and z; its radius within [R - wn, sqrt((R + wn)^2 + wt^2)]
// and its phi within atan(wt / (R - wn)).  Each bound widened by 0.1 % plus
// 1e-6 rad / 1e-5 cm (the hits' bins are computed in float), mapped to eta
// rows e0..e1 and phi bins fa0..fa1 (+ fb0..fb1 across phi = +-pi).
__device__ void window_f64(const double p[6], const double C[21], double R, double v0, double v1, double v2,
                           double cut, double Si[6], int& e0, int& e1, int& fa0, int& fa1, int& fb0, int& fb1) {
  const double pi = 3.14159265358979323846;
  kf::inverse_S(C, v0, v1, v2, Si);
  const double X = p[0], Y = p[1], Z = p[2];
  const double rr = sqrt(X * X + Y * Y);
  const double cph = X / rr, sph = Y / rr;
  const double s00 = C[0] + v0, s10 = C[1], s11 = C[2] + v1, s22 = C[5] + v2;
  const double Stt = sph * sph * s00 - 2.0 * sph * cph * s10 + cph * cph * s11;
  const double Snn = cph * cph * s00 + 2.0 * sph * cph * s10 + sph * sph * s11;
  const double wt = sqrt(cut * fmax(Stt, 0.0)), wn = sqrt(cut * fmax(Snn, 0.0)), wz = sqrt(cut * fmax(s22, 0.0));
  const double widen = 1.001;
  fa0 = 0;
  fa1 = KF_BIN_PHI - 1;
  fb0 = 0;
  fb1 = -1;
  const double rin = R - wn * widen;
  const double phic = atan2(Y, X);
  const double dphi = (rin > 0.5 * R && wt * widen < rin) ? atan(wt * widen / rin) * widen + 1e-6 : 10.0;
  if (dphi < 1.0) {
    const double scale = double(KF_BIN_PHI) / (2.0 * pi);
    const int f0 = int(floor((phic - dphi + pi) * scale)), f1 = int(floor((phic + dphi + pi) * scale));
    if (f1 - f0 + 1 < KF_BIN_PHI) {
      if (f0 < 0) {
        fa0 = f0 + KF_BIN_PHI;
        fb0 = 0;
        fb1 = f1;
      } else if (f1 >= KF_BIN_PHI) {
        fa0 = f0;
        fb0 = 0;
        fb1 = f1 - KF_BIN_PHI;
      } else {
        fa0 = f0;
        fa1 = f1;
      }
    }
  }
  e0 = 0;
  e1 = KF_BIN_ETA - 1;
  const double rlo = R - wn * widen - 1e-5;
  const double rhi = sqrt((R + wn) * (R + wn) + wt * wt) * widen + 1e-5;
  if (rlo > 0.0) {
    const double zlo = Z - wz * widen - 1e-5, zhi = Z + wz * widen + 1e-5;
    const double tmin = zlo >= 0.0 ? zlo / rhi : zlo / rlo;
    const double tmax = zhi >= 0.0 ? zhi / rlo : zhi / rhi;
    e0 = eta_bin64(asinh(tmin));
    e1 = eta_bin64(asinh(tmax));
  }
}

__global__ void __launch_bounds__(kF64Threads) build_f64_step_kernel(const StepF64Args A) {
  const int64_t j = A.begin + int64_t(blockIdx.x) * kF64Threads + threadIdx.x;
  if (j >= A.end) return;
  const int64_t SM = A.S * A.max_cands;
  const int nc = A.in.ncand[j];
  const double a = A.a_scale * double(A.charge[j]);
  const int64_t h0 = A.seg_off[A.seg];
  const int32_t* boff = A.bin_off + int64_t(A.seg) * (KF_NBINS + 1);
  // the parents' predictions (local memory) and the seed's best children
  double pp[kF64MaxCands][6], pC[kF64MaxCands][21];
  int32_t pst[kF64MaxCands];
  bool pstop[kF64MaxCands];
  Child list[kF64MaxCands];
  int n_keep = 0;
  for (int c = 0; c < nc; ++c) {
    const int64_t slot = j * A.max_cands + c;
    double p[6], lo[3] = {0.0, 0.0, 0.0}, C[21];
    for (int w = 0; w < 6; ++w) p[w] = A.in.par[w * SM + slot];
    for (int w = 0; w < 21; ++w) C[w] = A.in.cov[w * SM + slot];
    const double chi2tot = A.in.chi2[slot];
    const int32_t meta = A.in.meta[slot];
    const int nh = meta & 0xff;
    int32_t st = meta >> 8;
    bool stopped = (st & KF_ST_STOPPED) != 0;
    if (!stopped) {
      const int r = kf::propagate<double, kNewtonBuild64, false>(p, lo, C, a, A.R);
      if (r) {
        st |= r;
        stopped = true;
      } else if (A.x_x0 > 0.0) {
        kf::scatter(p, lo, C, A.x_x0, A.mass);
      }
    }
    bool any = false;
    if (!stopped) {
      double Si[6];
      int e0, e1, fa0, fa1, fb0, fb1;
      window_f64(p, C, A.R, A.v0, A.v1, A.v2, A.cut, Si, e0, e1, fa0, fa1, fb0, fb1);
      for (int er = e0; er <= e1; ++er)
        for (int part = 0; part < 2; ++part) {
          const int f0 = part ? fb0 : fa0, f1 = part ? fb1 : fa1;
          if (f1 < f0) continue;
          const int u0 = boff[er * KF_BIN_PHI + f0], u1 = boff[er * KF_BIN_PHI + f1 + 1];
          for (int u = u0; u < u1; ++u) {
            const float4 m = A.hits[h0 + u];
            const double r0 = double(m.x) - p[0], r1 = double(m.y) - p[1], r2 = double(m.z) - p[2];
            const double c2 = kf::chi2_of(r0, r1, r2, Si);
            const int id = __float_as_int(m.w);
            if (c2 < A.cut && id < KF_MAX_HITS_PER_SEGMENT) {
              keep_child(list, n_keep, A.max_cands, Child{nh + 1, chi2tot + c2, c, id, u});
              any = true;
            }
          }
        }
    }
    // no compatible hit (or a stopped candidate): one child without a hit
    if (!any) keep_child(list, n_keep, A.max_cands, Child{nh, chi2tot, c, -1, -1});
    for (int w = 0; w < 6; ++w) pp[c][w] = p[w];
    for (int w = 0; w < 21; ++w) pC[c][w] = C[w];
    pst[c] = st;
    pstop[c] = stopped;
  }
  // clone engine: copy and update only the kept children
  for (int r = 0; r < n_keep; ++r) {
    const Child& ch = list[r];
    double q[6], ql[3] = {0.0, 0.0, 0.0}, qC[21];
    for (int w = 0; w < 6; ++w) q[w] = pp[ch.parent][w];
    for (int w = 0; w < 21; ++w) qC[w] = pC[ch.parent][w];
    int32_t st = pst[ch.parent];
    if (ch.hit >= 0) {
      const float4 m = A.hits[h0 + ch.pos];
      double Si[6];
      kf::inverse_S(qC, A.v0, A.v1, A.v2, Si);
      double r0, r1, r2;
      kf::residual<double, false>(q, ql, double(m.x), double(m.y), double(m.z), r0, r1, r2);
      kf::kalman_update<double, false>(q, ql, qC, Si, r0, r1, r2, A.v0, A.v1, A.v2);
    } else if (!pstop[ch.parent]) {
      st |= KF_ST_NO_HIT;
    }
    const int64_t slot = j * A.max_cands + r;
    for (int w = 0; w < 6; ++w) A.out.par[w * SM + slot] = q[w];
    for (int w = 0; w < 21; ++w) A.out.cov[w * SM + slot] = qC[w];
    A.out.chi2[slot] = ch.chi2;
    A.out.meta[slot] = ch.nh | (st << 8);
    A.hist_parent[slot] = int8_t(ch.parent);
    A.hist_hit[slot] = ch.hit;
  }
  A.out.ncand[j] = int8_t(n_keep);
}

struct InitF64Args {
  CandF64 out;
  const double* par;
  const double* cov;
  int64_t S;
  int max_cands;
};

__global__ void build_f64_init_kernel(const InitF64Args A) {
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= A.S) return;
  const int64_t SM = A.S * A.max_cands, slot = j * A.max_cands;
  for (int w = 0; w < 6; ++w) A.out.par[w * SM + slot] = A.par[w * A.S + j];
  for (int w = 0; w < 21; ++w) A.out.cov[w * SM + slot] = A.cov[w * A.S + j];
  A.out.chi2[slot] = 0.0;
  A.out.meta[slot] = 0;
  A.out.ncand[j] = 1;
}

struct FinalF64Args {
  CandF64 cand;
  const int8_t* hist_parent;  // [L][SM]
  const int32_t* hist_hit;    // [L][SM]
  int64_t S;
  int n_layers, max_cands;
  kf_build_result_f64 out;
};

__device__ bool pd5_f64(const double p[6], const double C[21]) {
  using kf::sym;
  const double r = sqrt(p[0] * p[0] + p[1] * p[1]);
  const double t0 = r > 0.0 ? -p[1] / r : 0.0, t1 = r > 0.0 ? p[0] / r : 1.0;
  double M[5][5], Lc[5][5];
  M[0][0] = t0 * t0 * C[sym(0, 0)] + 2.0 * t0 * t1 * C[sym(1, 0)] + t1 * t1 * C[sym(1, 1)];
  for (int a = 1; a < 5; ++a) {
    M[a][0] = t0 * C[sym(0, a + 1)] + t1 * C[sym(1, a + 1)];
    for (int b = 1; b <= a; ++b) M[a][b] = C[sym(a + 1, b + 1)];
  }
  for (int a = 0; a < 5; ++a) {
    double d = M[a][a];
    for (int b = 0; b < a; ++b) d -= Lc[a][b] * Lc[a][b];
    if (!(d > 0.0)) return false;
    Lc[a][a] = sqrt(d);
    for (int i = a + 1; i < 5; ++i) {
      double v = M[i][a];
      for (int b = 0; b < a; ++b) v -= Lc[i][b] * Lc[a][b];
      Lc[i][a] = v / Lc[a][a];
    }
  }
  return true;
}

__global__ void build_f64_final_kernel(const FinalF64Args A) {
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= A.S) return;
  const int64_t SM = A.S * A.max_cands, slot = j * A.max_cands;  // rank 0: the best candidate
  double p[6], C[21];
  for (int w = 0; w < 6; ++w) p[w] = A.cand.par[w * SM + slot];
  for (int w = 0; w < 21; ++w) C[w] = A.cand.cov[w * SM + slot];
  const kf_build_result_f64& o = A.out;
  for (int w = 0; w < 6; ++w) o.best.par[w * A.S + j] = p[w];
  for (int w = 0; w < 21; ++w) o.best.cov[w * A.S + j] = C[w];
  const int32_t meta = A.cand.meta[slot];
  int32_t st = meta >> 8;
  if (!pd5_f64(p, C)) st |= KF_ST_NOT_PD;
  if (o.chi2_tot) o.chi2_tot[j] = A.cand.chi2[slot];
  if (o.n_hits) o.n_hits[j] = meta & 0xff;
  if (o.status) o.status[j] = st;
  if (o.hit_idx) {
    int k = 0;
    for (int l = A.n_layers - 1; l >= 0; --l) {
      const int64_t h = int64_t(l) * SM + j * A.max_cands + k;
      o.hit_idx[int64_t(l) * A.S + j] = A.hist_hit[h];
      k = A.hist_parent[h];
    }
  }
}

size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

size_t cand_f64_bytes(int64_t SM, int64_t S) {
  return al256(size_t(SM) * 27 * sizeof(double)) + al256(size_t(SM) * sizeof(double)) +
         al256(size_t(SM) * sizeof(int32_t)) + al256(size_t(S));
}

CandF64 cand_f64_at(char* q, int64_t SM, int64_t S) {
  CandF64 c;
  c.par = reinterpret_cast<double*>(q);
  c.cov = c.par + 6 * SM;
  q += al256(size_t(SM) * 27 * sizeof(double));
  c.chi2 = reinterpret_cast<double*>(q);
  q += al256(size_t(SM) * sizeof(double));
  c.meta = reinterpret_cast<int32_t*>(q);
  q += al256(size_t(SM) * sizeof(int32_t));
  c.ncand = reinterpret_cast<int8_t*>(q);
  (void)S;
  return c;
}

}  // namespace
}  // namespace kfi

using namespace kfi;

extern "C" int kf_build_f64(kf_ctx* ctx, const kf_tracks_f64* seeds, const int64_t* event_off,
                            const kf_layer_hit_bins* bins, int32_t max_cands, kf_build_result_f64* out,
                            void* stream) {
  if (!ctx || !seeds || !event_off || !bins || !out) return KF_EINVAL;
  if (max_cands < 1 || max_cands > kF64MaxCands) return KF_EINVAL;
  if (seeds->n < 0 || bins->n_events < 1 || bins->n_layers < 1 || bins->first_layer < 0 ||
      bins->first_layer + bins->n_layers > ctx->cfg.n_layers)
    return KF_EINVAL;
  const int64_t S = seeds->n;
  const int E = bins->n_events;
  if (event_off[0] != 0 || event_off[E] != S) return KF_EINVAL;
  for (int e = 0; e < E; ++e)
    if (event_off[e + 1] < event_off[e]) return KF_EINVAL;
  if (S == 0) return KF_OK;
  if (!seeds->par || !seeds->cov || !seeds->charge || !bins->bin_off || !bins->seg_off) return KF_EINVAL;
  if (bins->n_hits > 0 && !bins->hits) return KF_EINVAL;
  if (!out->best.par || !out->best.cov) return KF_EINVAL;
  KF_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  const int L = bins->n_layers;
  const int64_t SM = S * max_cands;
  const size_t b_cand = cand_f64_bytes(SM, S);
  const size_t b_hp = al256(size_t(L) * SM), b_hh = al256(size_t(L) * SM * sizeof(int32_t));
  int rc = scratch_reserve(ctx, ctx->s_build64, 2 * b_cand + b_hp + b_hh);
  if (rc) return rc;
  char* base = static_cast<char*>(ctx->s_build64.ptr);
  CandF64 buf[2] = {cand_f64_at(base, SM, S), cand_f64_at(base + b_cand, SM, S)};
  int8_t* hist_parent = reinterpret_cast<int8_t*>(base + 2 * b_cand);
  int32_t* hist_hit = reinterpret_cast<int32_t*>(base + 2 * b_cand + b_hp);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  InitF64Args ia{buf[0], seeds->par, seeds->cov, S, max_cands};
  build_f64_init_kernel<<<int((S + 255) / 256), 256, 0, st>>>(ia);
  KF_CUDA_TRY(ctx, cudaGetLastError());
  const double sxy = ctx->cfg.sigma_xy_cm, sz = ctx->cfg.sigma_z_cm;
  for (int l = 0; l < L; ++l) {
    for (int e = 0; e < E; ++e) {
      const int64_t b = event_off[e], en = event_off[e + 1];
      if (en <= b) continue;
      StepF64Args a;
      a.in = buf[l & 1];
      a.out = buf[(l + 1) & 1];
      a.hist_parent = hist_parent + int64_t(l) * SM;
      a.hist_hit = hist_hit + int64_t(l) * SM;
      a.charge = seeds->charge;
      a.hits = reinterpret_cast<const float4*>(bins->hits);
      a.bin_off = bins->bin_off;
      a.seg_off = bins->seg_off;
      a.S = S;
      a.begin = b;
      a.end = en;
      a.seg = e * L + l;
      a.max_cands = max_cands;
      a.a_scale = kCLight * double(ctx->cfg.bz_tesla);
      a.R = double(ctx->radius[bins->first_layer + l]);
      a.x_x0 = double(ctx->x_x0[bins->first_layer + l]);
      a.mass = double(ctx->mass);
      a.v0 = a.v1 = sxy * sxy;
      a.v2 = sz * sz;
      a.cut = double(ctx->cfg.chi2_cut);
      build_f64_step_kernel<<<int((en - b + kF64Threads - 1) / kF64Threads), kF64Threads, 0, st>>>(a);
      KF_CUDA_TRY(ctx, cudaGetLastError());
    }
  }
  FinalF64Args fa{buf[L & 1], hist_parent, hist_hit, S, L, max_cands, *out};
  build_f64_final_kernel<<<int((S + 127) / 128), 128, 0, st>>>(fa);
  KF_CUDA_TRY(ctx, cudaGetLastError());
  return KF_OK;
}
