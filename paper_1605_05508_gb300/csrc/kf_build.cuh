// kf_build.cuh -- candidate buffers, slot table and launchers of the
// clone-engine build kernels (kf_build.cu), shared with the serving loop.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/kf.h"
#include "kf_internal.h"

namespace kfi {

constexpr int kGroup = 8;           // lanes (candidate slots) per seed
constexpr int kBuildThreads = 128;  // 16 seeds per block
constexpr int kBuildBlocksPerSM = 5;  // resident blocks of kBuildThreads (96 registers a thread)
constexpr int kNewtonBuild = 12;
constexpr int kBuildTile = 512;     // hits staged per warp when hit staging is on
constexpr int kPackSeeds = 128;     // seeds per block of the candidate-packed step (scan scheme 2)
constexpr int kParN = 9;  // x y z px py pz + low parts of x y z
constexpr uint64_t kNoKey = ~0ull;
constexpr unsigned kFull = 0xffffffffu;

// Candidate k (0 .. kGroup-1, by rank) of seed j among S seeds.  Rank-major
// (k S + j: the candidates of one rank contiguous over the seeds) suits a
// buffer with one or two candidates a seed, whose loads and stores then fill
// whole 32-byte sectors; seed-major (kGroup j + k: a seed's candidates in one
// sector) suits a buffer with five or six.
__host__ __device__ __forceinline__ int64_t cand_slot(int64_t j, int k, int64_t S, bool rank_major) {
  return rank_major ? int64_t(k) * S + j : j * kGroup + k;
}
// Buffer b of a build holds the candidates after b building layers (b = 0:
// the seeds).  Buffers b < rank_major_buffers(...) are rank-major, the rest
// seed-major: with max_cands <= 2 every buffer, otherwise the seeds and the
// first layer's children (one to three candidates a seed).
inline int rank_major_buffers(int max_cands, int n_layers) { return max_cands <= 2 ? n_layers + 1 : 2; }

struct CandBuf {
  float* par;      // [9][S8], S8 = kGroup * S, slot cand_slot(j, k, S, layout)
  float* cov;      // [21][S8]
  float* chi2;     // [S8] chi2_tot
  int32_t* meta;   // [S8] nHits | status << 8
  int8_t* ncand;   // [S]
};

// One independent group of seeds advanced by a build step: a whole batch
// (kf_build) or one served event (kf_serve).  Slots of one launch may sit at
// different layers.  Blocks [block_begin, next slot's block_begin) serve it.
struct BuildSlot {
  CandBuf in, out;
  int8_t* hist_parent;       // [S8] of this layer (slots in the layout of `out`)
  int32_t* hist_hit;         // [S8] of this layer
  const int32_t* seed_evt;   // [S] sorted position -> event, or null (event 0)
  const int32_t* seed_perm;  // [S] sorted position -> seed index, or null (the identity)
  const int8_t* charge;      // [S] by seed index
  const float4* hits;
  const int32_t* bin_off;
  const int64_t* seg_off;
  int64_t S;
  int layer, n_layers;
  float R;
  float x_x0;  // this layer's thickness in radiation lengths (0: none)
  int in_rm, out_rm;  // 1: `in` / `out` (and the history) are rank-major (cand_slot)
  int block_begin;
};

struct BuildStepArgs {
  const BuildSlot* slots;  // device table
  int n_slots, max_cands;
  float a_scale, v0, v1, v2, cut;
  float mass;            // particle mass of the scattering model
  int pack_seeds;        // candidate-packed layouts: seeds per block (<= the block's threads; 0: as many)
  int layers;            // candidate-packed layouts: > 1 = `slots` are that many consecutive layers of
                         // one batch and each block takes its seeds through all of them
  // test hook (kf_test_build_stage_fault), grouped layouts with hit staging:
  // the warp of this index in the launch issues no copies and arms nothing,
  // and the waits for staged hits give up after test_wait_limit polls (0: the
  // normal limit)
  int64_t test_skip_warp = -1;
  uint32_t test_wait_limit = 0;
};

struct BuildInitArgs {
  CandBuf out;
  const float* par;
  const float* lo;
  const float* cov;
  const int32_t* seed_perm;
  int64_t n;  // seeds (stride of the seed arrays)
  int64_t S;
};

struct BuildFinalArgs {
  CandBuf cand;
  const int8_t* hist_parent;  // [L][S8]
  const int32_t* hist_hit;    // [L][S8]
  const int32_t* seed_perm;  // or null (the identity)
  int64_t S;
  int n_layers, max_cands;
  int rm_buffers;  // rank_major_buffers(max_cands, n_layers)
  int paths_only;  // 1: only the paths (hit_idx, cand_hit_idx; of cand only ncand is read),
                   // 2: also the best covariance check (status; cand: ncand, rank 0's low part)
  kf_build_result out;
};

// Candidate buffer of S seeds at `base` (256-byte aligned pieces).
inline size_t cand_piece(int64_t S) { return (size_t(S) * kGroup * 4 + 255) & ~size_t(255); }
inline size_t cand_bytes(int64_t S) { return (kParN + 23) * cand_piece(S) + ((size_t(S) + 255) & ~size_t(255)); }
inline CandBuf cand_at(char* q, int64_t S) {
  const size_t pc = cand_piece(S);
  CandBuf c;
  c.par = reinterpret_cast<float*>(q);
  c.cov = reinterpret_cast<float*>(q + kParN * pc);
  c.chi2 = reinterpret_cast<float*>(q + (kParN + 21) * pc);
  c.meta = reinterpret_cast<int32_t*>(q + (kParN + 22) * pc);
  c.ncand = reinterpret_cast<int8_t*>(q + (kParN + 23) * pc);
  return c;
}

// tile: 0 (scan global memory) or kBuildTile (stage the window hits per
// warp); list: 4 (lane lists of 4 children, when max_cands <= 4) or 8;
// scan: 0 (each lane scans its own candidate's window), 1 (the seed's
// lanes scan each parent's window together), 2 or 3 (candidate-packed, 128 or
// 64 seeds per block: grid of build_step_blocks(S, scan); tile is ignored)
cudaError_t launch_build_step(const BuildStepArgs& a, int grid, cudaStream_t st, int tile, int list, int scan);
// Seeds (threads) per block of the candidate-packed layouts: scan 2: 128,
// scan 3: 64; 0 for the other layouts.
inline int packed_seeds_per_block(int scan) { return scan == 2 ? kPackSeeds : scan == 3 ? kPackSeeds / 2 : 0; }
inline bool is_packed(int scan) { return packed_seeds_per_block(scan) > 0; }

// Blocks of the build step for S seeds: 8 lanes per seed, 16 seeds per block,
// or one seed per thread in the candidate-packed layouts.
inline int build_step_blocks(int64_t S, int scan) {
  const int per_block = is_packed(scan) ? packed_seeds_per_block(scan) : kBuildThreads / kGroup;
  return int((S + per_block - 1) / per_block);
}

// Candidate-packed steps that keep more than two candidates a seed: seeds per
// block so that `seeds` spread over a whole number of waves of resident blocks
// (a block's several rounds take about equal time, so a last partial wave
// would leave most SMs idle at the end of the step); 0 otherwise (one or two
// candidates: a block's single round is short and a full block of seeds keeps
// its threads busier).
inline int build_pack_seeds(int64_t seeds, int scan, int max_cands, int num_sms) {
  if (!is_packed(scan) || max_cands <= 2 || num_sms <= 0 || seeds <= 0) return 0;
  const int per_block = packed_seeds_per_block(scan);
  const int64_t wave = int64_t(num_sms) * kBuildBlocksPerSM * (kPackSeeds / per_block);
  const int64_t waves = ((seeds + per_block - 1) / per_block + wave - 1) / wave;
  return int((seeds + waves * wave - 1) / (waves * wave));
}
// Register-resident build (thread layout 4, build_resident_kernel): each warp
// takes groups of 32 / W seeds, W lanes a seed (W >= max_cands, one candidate
// slot a lane), through building layers l0 .. n_layers-1 with every
// candidate's state in registers; it reads buffer l0 and writes only the
// per-layer history and buffer n_layers.
constexpr int kResThreads = 128;
constexpr int kResBlocksPerSM = 4;
// resident blocks per SM of build_resident_kernel<W>: 4 (128 registers a
// thread); with one lane a seed 5 (measured: 3 % faster there, 6 % slower
// at W = 6, where the registers are needed)
constexpr int resident_blocks_per_sm(int W) { return W == 1 ? 5 : kResBlocksPerSM; }
// One batch of seeds of a register-resident build: the whole batch of a
// kf_build call, or one served event.
struct ResidentBatch {
  CandBuf in;                // buffer l0 (layout in_rm)
  CandBuf out;               // buffer n_layers (layout out_rm); must not alias `in`
  int8_t* hist_parent;       // [n_layers][S8]: layer l's slots in the layout of buffer l + 1
  int32_t* hist_hit;         // [n_layers][S8]
  const int32_t* seed_evt;   // [S] sorted position -> event, or null (event 0)
  const int32_t* seed_perm;  // [S] sorted position -> seed index, or null (the identity)
  const int8_t* charge;      // [S] by seed index
  const float4* hits;
  const int32_t* bin_off;
  const int64_t* seg_off;
  // the segments' sub-bin starts ([n_seg][KF_NBINS_FINE + 1]), or null: the
  // windows then look up the bins of bin_off
  const int32_t* fine_off;
  int64_t S;
  int64_t group_begin;       // with a table: the launch's first group of this batch
  int64_t seed_begin;        // with a table: the first-layer launch's first seed of this batch
  // the seeds themselves ([6] / [3] (or null: zero) / [21] x S, by seed
  // index), read in place of buffer `in` when set (then l0 = 0: every seed
  // one candidate, chi2 0, no hit)
  const float* seed_par;
  const float* seed_lo;
  const float* seed_cov;
  // the final selection, done by the kernel after the last layer when
  // res.best.par is set (the best candidate and the optional per-candidate
  // summaries, as build_final_kernel writes them, all but the paths; only
  // out.ncand is then written); else the candidates go to `out`
  kf_build_result res;
};
struct BuildResidentArgs {
  ResidentBatch one;                 // the batch, when `table` is null
  const ResidentBatch* table;        // device table of n_batches batches (served events), or null
  int n_batches;
  int64_t n_groups;                  // with a table: groups of all its batches
  int64_t n_seeds;                   // with a table: seeds of all its batches
  int n_layers, l0, rm_buffers, max_cands;
  int in_rm, out_rm;
  float a_scale, v0, v1, v2, cut, mass;
  float R[kMaxLayers];     // building layer radii
  float x_x0[kMaxLayers];  // building layer thickness in radiation lengths (0: none)
  // device counter, zero at launch: the warps fetch their next seed group
  // from it (build_resident_kernel)
  unsigned long long* group_counter;
};
// Lanes per seed of the resident layout for max_cands (1, 2, 4, 6 or 8).
inline int resident_lanes(int max_cands) {
  return max_cands <= 2 ? max_cands : max_cands <= 4 ? 4 : max_cands <= 6 ? 6 : 8;
}
// With several lanes a seed, the resident layout leaves the best covariance's
// positive-definiteness check to the final kernel (paths_only = 2).
inline bool resident_defers_pd(int max_cands) { return resident_lanes(max_cands) > 1; }
// seeds per warp group of the resident layout (32 / lanes per seed)
inline int resident_group(int max_cands) { return 32 / resident_lanes(max_cands); }
cudaError_t launch_build_resident(const BuildResidentArgs& a, int num_sms, cudaStream_t st);
cudaError_t launch_build_first_layer(const BuildResidentArgs& a, cudaStream_t st);

cudaError_t launch_build_init(const BuildInitArgs& a, cudaStream_t st);
cudaError_t launch_build_final(const BuildFinalArgs& a, cudaStream_t st);

}  // namespace kfi
