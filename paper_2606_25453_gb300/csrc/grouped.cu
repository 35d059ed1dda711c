// grouped.cu -- many independent Scheme I products in one persistent launch.
//
// The paper has no batched interface; this follows its tile model (Table I):
// each product is cut into output tiles of the configuration its shape
// bucket was tuned to -- a tile shape (BM x BN: 64 x 32, 32 x 32 or 32 x 64,
// warps of 16 x 16) and a slice-pair schedule of the triangle (B-slice-major
// or A-slice-major) --; the tiles of one configuration form one work list, balanced over the CTAs by a
// longest-processing-time assignment (tile cost = number of K chunks), and
// one persistent kernel per configuration in use walks each CTA's list.  The
// exponent scan and the split of all operands are one launch each.  The
// launch sequence (memset, scan, split, then the GEMM launches on parallel
// branches, so that one kernel fills the tail of another's) is
// captured once into a CUDA graph and replayed while the product
// descriptors stay identical.  A timing autotuner picks the configuration
// per shape bucket (log2 classes of sqrt(M N) and of K) by coordinate
// descent on the time of the whole batch.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <queue>
#include <sstream>
#include <string>
#include <vector>

#include "emu_handle.h"
#include "emu_internal.h"
#include "gemm_I_core.cuh"
#include "split_core.cuh"

namespace emu {

namespace {

struct GProb {
  const double* A;
  const double* B;
  double* C;
  int64_t lda, ldb, ldc;
  int M, N, K, nk32;
  double alpha, beta;
  unsigned long long* maxA;
  unsigned long long* maxB;
  int32_t* EA;
  int32_t* FB;
  int8_t* hatA;
  int8_t* hatB;
  int64_t rows_a, rows_b, nchunks;
};

// True when the rows of a row-major binary64 matrix start on 16-byte
// boundaries (base aligned, even leading dimension).
__device__ __forceinline__ bool a16(const double* X, int64_t ld) {
  return ((reinterpret_cast<uintptr_t>(X) & 15u) | static_cast<uintptr_t>(ld & 1)) == 0;
}

// index of the problem owning block `blk` in a prefix array start[0..count]
__device__ __forceinline__ int find_prob(const int* start, int count, int blk) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (start[mid] <= blk) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------------------------------- scan
// Blocks [0, startA[count]) scan rows of A (one warp per row, K segments of
// 2048); the rest scan columns of B (32 columns x 8 K-lanes, segments of 256).
__global__ void grouped_scan_kernel(const GProb* __restrict__ probs, int count, const int* __restrict__ startA,
                                    const int* __restrict__ startB, int* status) {
  int blk = blockIdx.x;
  const int totA = startA[count];
  if (blk < totA) {
    int pi = find_prob(startA, count, blk);
    const GProb& pr = probs[pi];
    int local = blk - startA[pi];
    int kseg = (pr.K + 2047) / 2048;
    int rb = local / kseg, ks = local % kseg;
    int lane = threadIdx.x & 31;
    int r = rb * 8 + (threadIdx.x >> 5);
    if (r >= pr.M) return;
    int h0 = ks * 2048, h1 = min(h0 + 2048, pr.K);
    const double* row = pr.A + static_cast<int64_t>(r) * pr.lda;
    uint64_t mx = 0;
    int h = h0 + lane;
    if (a16(pr.A, pr.lda)) {  // 16-byte loads of element pairs (h0 is even)
      const uint4* pv = reinterpret_cast<const uint4*>(row + h0);
      const int nv = (h1 - h0) >> 1;
#pragma unroll 4
      for (int i = lane; i < nv; i += 32) {
        const uint4 v = __ldg(pv + i);
        const uint64_t x = ((static_cast<uint64_t>(v.y) << 32) | v.x) & 0x7FFFFFFFFFFFFFFFull;
        const uint64_t y = ((static_cast<uint64_t>(v.w) << 32) | v.z) & 0x7FFFFFFFFFFFFFFFull;
        mx = x > mx ? x : mx;
        mx = y > mx ? y : mx;
      }
      h = h0 + 2 * nv + lane;  // the odd last element, if any
    }
#pragma unroll 4
    for (; h < h1; h += 32) {
      uint64_t v = dbits(__ldg(row + h)) & 0x7FFFFFFFFFFFFFFFull;
      mx = v > mx ? v : mx;
    }
    for (int o = 16; o; o >>= 1) {
      uint64_t w = __shfl_xor_sync(0xffffffffu, mx, o);
      mx = w > mx ? w : mx;
    }
    if (lane == 0 && h0 < h1) {
      atomicMax(pr.maxA + r, static_cast<unsigned long long>(mx));
      if (mx >= 0x7FF0000000000000ull) set_status(status, ST_NONFINITE);
    }
    return;
  }
  blk -= totA;
  int pi = find_prob(startB, count, blk);
  const GProb& pr = probs[pi];
  int local = blk - startB[pi];
  int kseg = (pr.K + 255) / 256;
  int cb = local / kseg, ks = local % kseg;
  int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  int c = cb * 32 + tx;
  int h0 = ks * 256, h1 = min(h0 + 256, pr.K);
  uint64_t mx = 0;
  if (c < pr.N) {
#pragma unroll 4
    for (int h = h0 + ty; h < h1; h += 8) {
      uint64_t v = dbits(__ldg(pr.B + static_cast<int64_t>(h) * pr.ldb + c)) & 0x7FFFFFFFFFFFFFFFull;
      mx = v > mx ? v : mx;
    }
  }
  __shared__ uint64_t red[8][32];
  red[ty][tx] = mx;
  __syncthreads();
  if (ty == 0 && c < pr.N && h0 < h1) {
    for (int q = 1; q < 8; ++q) mx = red[q][tx] > mx ? red[q][tx] : mx;
    atomicMax(pr.maxB + c, static_cast<unsigned long long>(mx));
    if (mx >= 0x7FF0000000000000ull) set_status(status, ST_NONFINITE);
  }
}

// ---------------------------------------------------------------- split
__device__ __forceinline__ int exp_of(const unsigned long long* mb, int r, int rows) {
  if (r >= rows) return 0;
  uint64_t v = mb[r];
  return v >= 0x7FF0000000000000ull ? 0 : frexp_exp_bits(v);
}

// Blocks [0, startA[count]): A rows, one warp per (row, group of four
// 32-wide K-chunks); lane l packs elements 4l .. 4l+3 of the group into one
// word per slice.  The rest: B columns, a block per (32 columns, 128 K
// elements), read coalesced along the row of B into shared memory and then
// packed the same way (the layout of the dense strided split).
template <int P>
__global__ void __launch_bounds__(256) grouped_split_kernel(const GProb* __restrict__ probs, int count,
                                                            const int* __restrict__ startA,
                                                            const int* __restrict__ startB) {
  __shared__ uint64_t tile[32][133];
  int blk = blockIdx.x;
  const int totA = startA[count];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (blk < totA) {
    const int pi = find_prob(startA, count, blk);
    const GProb& pr = probs[pi];
    const int64_t ngroups = (pr.nchunks + 3) / 4;
    const int64_t w = static_cast<int64_t>(blk - startA[pi]) * 8 + warp;
    if (w >= pr.rows_a * ngroups) return;
    const int r = static_cast<int>(w / ngroups);
    const int64_t c = (w % ngroups) * 4 + (lane >> 3);
    if (c >= pr.nchunks) return;
    const int64_t h0 = c * 32 + (lane & 7) * 4;
    const int E = exp_of(pr.maxA, r, pr.M);
    uint64_t bits[4];
    load4_kcontig(pr.A + static_cast<int64_t>(r < pr.M ? r : 0) * pr.lda, h0, pr.K, r < pr.M, a16(pr.A, pr.lda),
                  bits);
    uint32_t word[P];
    pack4<P, false>(bits, E, word);
    uint8_t* row = reinterpret_cast<uint8_t*>(pr.hatA) + static_cast<int64_t>(r) * pr.nchunks * 32 * P;
#pragma unroll
    for (int t = 0; t < P; ++t) *reinterpret_cast<uint32_t*>(row + (c * P + t) * 32 + (lane & 7) * 4) = word[t];
    if (c == 0 && lane == 0 && r < pr.M) pr.EA[r] = E;
    return;
  }
  blk -= totA;
  const int pi = find_prob(startB, count, blk);
  const GProb& pr = probs[pi];
  const int64_t ngroups = (pr.nchunks + 3) / 4;
  const int local = blk - startB[pi];
  const int64_t g = local % ngroups;
  const int64_t r0 = static_cast<int64_t>(local / ngroups) * 32;
  fill_tile_strided(tile, pr.B, pr.ldb, pr.N, pr.K, r0, g * 128, a16(pr.B, pr.ldb));
  __syncthreads();
  const int64_t c = g * 4 + (lane >> 3);
  for (int rl = warp; rl < 32; rl += 8) {
    const int64_t r = r0 + rl;
    if (r >= pr.rows_b || c >= pr.nchunks) continue;
    const int E = exp_of(pr.maxB, static_cast<int>(r), pr.N);
    uint64_t bits[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) bits[q] = tile[rl][q * 33 + lane];
    uint32_t word[P];
    pack4<P, false>(bits, E, word);
    uint8_t* row = reinterpret_cast<uint8_t*>(pr.hatB) + r * pr.nchunks * 32 * P;
#pragma unroll
    for (int t = 0; t < P; ++t) *reinterpret_cast<uint32_t*>(row + (c * P + t) * 32 + (lane & 7) * 4) = word[t];
    if (c == 0 && lane == 0 && r < pr.N) pr.FB[r] = E;
  }
}

// ---------------------------------------------------------------- GEMM
template <int P, int BM, int BN, int SCHED>
struct CfgG {
  static constexpr int kWM = BM / 16, kWN = BN / 16, kCW = kWM * kWN;
  static constexpr int kThreads = (kCW + 1) * 32;
  static constexpr int kBlkA = BM * 32, kBlkB = BN * 32;
  static constexpr int kStageBytes = P * (kBlkA + kBlkB);
  static constexpr int kBudget = kCW >= 8 ? 163840 : 98304;  // 4-warp tiles run 2 CTAs per SM
  static constexpr int kRaw = kBudget / kStageBytes;
  static constexpr int kStages = kRaw < 2 ? 2 : (kRaw > 8 ? 8 : kRaw);
  static constexpr int kSmem = kStages * kStageBytes + 1024 + 2 * kStages * 8 + 64;
  static constexpr int kOcc = kCW >= 8 ? 1 : 2;
};

// SCHED: slice-pair order of the triangle, 0 = B-slice-major (TriAll),
// 1 = A-slice-major (TriAllByA).
template <int P, int BM, int BN, int SCHED>
__global__ void __launch_bounds__(CfgG<P, BM, BN, SCHED>::kThreads, CfgG<P, BM, BN, SCHED>::kOcc)
    gemm_I_grouped_kernel(const GProb* __restrict__ probs, const CUtensorMap* __restrict__ maps,
                          const int4* __restrict__ tiles, const int* __restrict__ cta_ptr, int kc32, int escale,
                          int* status) {
  using Cfg = CfgG<P, BM, BN, SCHED>;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* smem = smem_raw + (base - raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + Cfg::kStages * Cfg::kStageBytes);
  uint64_t* empty = full + Cfg::kStages;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < Cfg::kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], Cfg::kCW);
    }
    fence_mbar_init();
  }
  __syncthreads();
  const int t0 = cta_ptr[blockIdx.x], t1 = cta_ptr[blockIdx.x + 1];

  if (warp == Cfg::kCW) {
    if (lane == 0) {
      uint32_t it = 0;
      for (int t = t0; t < t1; ++t) {
        const int4 tl = tiles[t];
        const CUtensorMap* dA = maps + 2 * tl.x;
        const CUtensorMap* dB = dA + 1;
        const int nk32 = probs[tl.x].nk32;
        for (int kk = 0; kk < nk32; ++kk, ++it) {
          const uint32_t stage = it % Cfg::kStages;
          const uint32_t par = (it / Cfg::kStages) & 1u;
          if (it >= static_cast<uint32_t>(Cfg::kStages) && !mbar_wait_bounded(&empty[stage], par ^ 1u)) {
            set_status(status, ST_TIMEOUT);
            return;
          }
          mbar_arrive_expect_tx(&full[stage], Cfg::kStageBytes);
          uint8_t* sA = smem + stage * Cfg::kStageBytes;
          uint8_t* sB = sA + P * Cfg::kBlkA;
#pragma unroll
          for (int q = 0; q < P; ++q) tma_load_2d(sA + q * Cfg::kBlkA, dA, &full[stage], (kk * P + q) * 32, tl.y * BM);
#pragma unroll
          for (int q = 0; q < P; ++q) tma_load_2d(sB + q * Cfg::kBlkB, dB, &full[stage], (kk * P + q) * 32, tl.z * BN);
        }
      }
    }
    return;
  }

  const int wm = warp / Cfg::kWN, wn = warp % Cfg::kWN;  // this warp's 16 x 16 patch of the tile
  const uint32_t a_off = swz32(wm * 16 + (lane & 15), lane >> 4);
  const uint32_t b_off = swz32(wn * 16 + (lane & 7) + ((lane >> 4) << 3), (lane >> 3) & 1);
  uint32_t it = 0;
  for (int t = t0; t < t1; ++t) {
    const int4 tl = tiles[t];
    const GProb& pr = probs[tl.x];
    int32_t acc[P][2][4];
    __int128 S[2][4];
#pragma unroll
    for (int s = 0; s < P; ++s)
#pragma unroll
      for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[s][nt][q] = 0;
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int q = 0; q < 4; ++q) S[nt][q] = 0;
    int since = 0;
    const int nk32 = pr.nk32;
    // a patch wholly outside the product (ragged last tiles) does no MMAs;
    // its warp still takes part in the stage handshake
    const bool live = tl.y * BM + wm * 16 < pr.M && tl.z * BN + wn * 16 < pr.N;
    for (int kk = 0; kk < nk32; ++kk, ++it) {
      const uint32_t stage = it % Cfg::kStages;
      const uint32_t par = (it / Cfg::kStages) & 1u;
      if (!mbar_wait_bounded(&full[stage], par)) {
        set_status(status, ST_TIMEOUT);
        return;
      }
      if (live) {
        const uint32_t sA = base + stage * Cfg::kStageBytes;
        const uint32_t sB = sA + P * Cfg::kBlkA;
        uint32_t af[P][4];
#pragma unroll
        for (int i = 0; i < P; ++i) ldsm_x4(sA + i * Cfg::kBlkA + a_off, af[i][0], af[i][1], af[i][2], af[i][3]);
        if constexpr (SCHED == 0)
          TriAll<P, Cfg::kBlkB, false>::run(acc, af, sB, b_off);
        else
          TriAllByA<P, Cfg::kBlkB, false>::run(acc, af, sB, b_off);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[stage]);
      if (++since == kc32) {
        if (live) fold<P, false>(acc, S);
        since = 0;
      }
    }
    if (!live) continue;
    fold<P, false>(acc, S);
    const int row0 = tl.y * BM + wm * 16 + (lane >> 2);
    const int col0 = tl.z * BN + wn * 16 + (lane & 3) * 2;
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        int row = row0 + (q >> 1) * 8, col = col0 + nt * 8 + (q & 1);
        if (row < pr.M && col < pr.N) {
          double d = i128_to_double_rn(S[nt][q]);
          double r = scale2(d, pr.EA[row] + pr.FB[col] + escale);
          double* cp = pr.C + static_cast<int64_t>(row) * pr.ldc + col;
          *cp = blas_update(pr.alpha, r, pr.beta, pr.beta != 0.0 ? *cp : 0.0);
        }
      }
  }
}

// ---------------------------------------------------------------- host plan
// Candidate configurations: tile shape x slice-pair schedule (0-2
// B-slice-major, 3-5 the same shapes A-slice-major; launch_by_cfg maps them
// to kernel instantiations).
constexpr int kNumCfg = 6;
constexpr int kCfgBM[kNumCfg] = {64, 32, 32, 64, 32, 32};
constexpr int kCfgBN[kNumCfg] = {32, 32, 64, 32, 32, 64};

// Products are processed in up to three stages, in decreasing order of GEMM
// work per operand byte: each stage's GEMM launches run while the scan and
// split of the next stages proceed beside them.  Stage s ends where the
// cumulative GEMM work reaches kStageEnd[s] of the batch's.
constexpr int kMaxStages = 3;
constexpr double kStageEnd[kMaxStages - 1] = {0.15, 0.5};

// One GEMM launch of a plan: the tiles of every product of one stage whose
// bucket uses configuration `cfg`.
struct SubPlan {
  int cfg = 0, grid = 0, stage = 0;
  int4* d_tiles = nullptr;
  int* d_cta = nullptr;
};

// Scan and split launches of one stage: products [first, first + count) of
// the plan's (stage-ordered) problem table, with block prefix arrays of
// their own.
struct StagePlan {
  int first = 0, count = 0;
  int* d_startA_scan = nullptr;
  int* d_startB_scan = nullptr;
  int* d_startA_split = nullptr;
  int* d_startB_split = nullptr;
  int scan_blocks = 0, split_blocks = 0;
};

struct GroupPlan {
  std::vector<emu_gemm_desc_t> descs;
  std::vector<int> pcfg;  // configuration of each product (caller's order)
  int p = 0, count = 0;
  int max_stages = kMaxStages;  // the setting the plan was built for
  int nstages = 1;
  StagePlan stages[kMaxStages];
  std::vector<SubPlan> subs;
  void* dev = nullptr;  // one device buffer: probs, maps, tiles, cta_ptr, starts, workspace
  size_t dev_bytes = 0;
  GProb* d_probs = nullptr;  // stage order
  CUtensorMap* d_maps = nullptr;
  unsigned long long* d_max = nullptr;
  size_t max_bytes = 0;
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
};

constexpr int kMaxSubs = kMaxStages * kNumCfg;

struct GroupState {
  GroupPlan* plan = nullptr;
  std::map<std::string, int> tuned;  // shape bucket -> configuration index
  cudaStream_t capture = nullptr;
  cudaStream_t side[kMaxSubs] = {};  // branches of the captured graph
  cudaEvent_t fork[kMaxStages] = {}, join[kMaxSubs] = {};
};

void free_plan(GroupPlan* pl) {
  if (!pl) return;
  if (pl->exec) cudaGraphExecDestroy(pl->exec);
  if (pl->graph) cudaGraphDestroy(pl->graph);
  if (pl->dev) cudaFree(pl->dev);
  delete pl;
}

GroupState* state_of(emu_handle_s* h) {
  if (!h->grouped) h->grouped = new GroupState();
  return static_cast<GroupState*>(h->grouped);
}

bool same_plan(const GroupPlan* pl, const emu_gemm_desc_t* b, int count, int p, const std::vector<int>& pcfg,
               int stages) {
  if (!pl || pl->p != p || pl->max_stages != stages || static_cast<int>(pl->descs.size()) != count ||
      pl->pcfg != pcfg)
    return false;
  return std::memcmp(pl->descs.data(), b, sizeof(emu_gemm_desc_t) * count) == 0;
}

// Shape bucket of one product: p, and log2 classes of its output side
// sqrt(M N) (below 64, 128, 256, 512, and above) and of K (below 128, 256,
// 512, 1024, and above).
std::string bucket_of(const emu_gemm_desc_t& d, int p) {
  const double side = std::sqrt(static_cast<double>(d.m) * static_cast<double>(d.n));
  const int sc = std::min(4, std::max(0, static_cast<int>(std::floor(std::log2(side))) - 5));
  const int kc = std::min(4, std::max(0, static_cast<int>(std::floor(std::log2(static_cast<double>(d.k)))) - 6));
  char buf[48];
  std::snprintf(buf, sizeof(buf), "p%d_s%d_k%d", p, sc, kc);
  return buf;
}

// Tuning-map key of the stage setting for slice count p.
std::string stages_key(int p) {
  char buf[32];
  std::snprintf(buf, sizeof(buf), "p%d_stages", p);
  return buf;
}

// Maximum stage count for slice count p from the tuned map (kMaxStages
// where untuned).
int stages_of(const GroupState* gs, int p) {
  auto it = gs->tuned.find(stages_key(p));
  return it != gs->tuned.end() ? it->second : kMaxStages;
}

// Tile configuration of each product from the tuned map (0 where untuned).
std::vector<int> configs_of(const GroupState* gs, int count, const emu_gemm_desc_t* d, int p) {
  std::vector<int> c(count, 0);
  for (int i = 0; i < count; ++i) {
    auto it = gs->tuned.find(bucket_of(d[i], p));
    if (it != gs->tuned.end()) c[i] = it->second;
  }
  return c;
}

template <int P, int BM, int BN, int SCHED>
cudaError_t launch_gemm_grouped(const GroupPlan& pl, const SubPlan& sp, int* status, cudaStream_t st,
                                bool attrs_only) {
  using Cfg = CfgG<P, BM, BN, SCHED>;
  if (attrs_only)
    return cudaFuncSetAttribute(gemm_I_grouped_kernel<P, BM, BN, SCHED>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::kSmem);
  gemm_I_grouped_kernel<P, BM, BN, SCHED><<<sp.grid, Cfg::kThreads, Cfg::kSmem, st>>>(
      pl.d_probs, pl.d_maps, sp.d_tiles, sp.d_cta, static_cast<int>(host_chunk_len_I(P) / 32), -14 - 8 * (P - 1),
      status);
  return cudaGetLastError();
}

template <int P>
cudaError_t launch_by_cfg(const GroupPlan& pl, const SubPlan& sp, int* status, cudaStream_t st, bool attrs_only) {
  switch (sp.cfg) {
    case 0: return launch_gemm_grouped<P, 64, 32, 0>(pl, sp, status, st, attrs_only);
    case 1: return launch_gemm_grouped<P, 32, 32, 0>(pl, sp, status, st, attrs_only);
    case 2: return launch_gemm_grouped<P, 32, 64, 0>(pl, sp, status, st, attrs_only);
    case 3: return launch_gemm_grouped<P, 64, 32, 1>(pl, sp, status, st, attrs_only);
    case 4: return launch_gemm_grouped<P, 32, 32, 1>(pl, sp, status, st, attrs_only);
    default: return launch_gemm_grouped<P, 32, 64, 1>(pl, sp, status, st, attrs_only);
  }
}

cudaError_t launch_sub(const GroupPlan& pl, const SubPlan& sp, int* status, cudaStream_t st, bool attrs_only) {
  switch (pl.p) {
#define EMU_GG(PP) case PP: return launch_by_cfg<PP>(pl, sp, status, st, attrs_only);
    EMU_GG(1) EMU_GG(2) EMU_GG(3) EMU_GG(4) EMU_GG(5) EMU_GG(6)
    EMU_GG(7) EMU_GG(8) EMU_GG(9) EMU_GG(10) EMU_GG(11) EMU_GG(12)
#undef EMU_GG
    default: return cudaErrorInvalidValue;
  }
}

// Set the dynamic shared memory limit of the plan's GEMM instantiations
// (done before capture: it is not stream work).
cudaError_t prepare_attrs(const GroupPlan& pl) {
  for (const SubPlan& sp : pl.subs) {
    cudaError_t e = launch_sub(pl, sp, nullptr, nullptr, true);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int occupancy_of(int cfg) { return (kCfgBM[cfg] / 16) * (kCfgBN[cfg] / 16) >= 8 ? 1 : 2; }

// memset on `st`; then per stage its scan and split on `st` and its GEMM
// launches (one per configuration) on side branches that fork after that
// split, so that stage 0's GEMMs overlap stage 1's scan and split; every
// branch joins `st` before the end.
cudaError_t launch_group(const GroupPlan& pl, GroupState* gs, int* status, cudaStream_t st) {
  cudaMemsetAsync(pl.d_max, 0, pl.max_bytes, st);
  for (int s = 0; s < pl.nstages; ++s) {
    const StagePlan& sg = pl.stages[s];
    const GProb* probs = pl.d_probs + sg.first;
    if (sg.scan_blocks)
      grouped_scan_kernel<<<sg.scan_blocks, 256, 0, st>>>(probs, sg.count, sg.d_startA_scan, sg.d_startB_scan,
                                                           status);
    if (sg.split_blocks) {
      switch (pl.p) {
#define EMU_GS(PP)                                                                                  \
  case PP:                                                                                          \
    grouped_split_kernel<PP><<<sg.split_blocks, 256, 0, st>>>(probs, sg.count, sg.d_startA_split, \
                                                               sg.d_startB_split);                 \
    break;
        EMU_GS(1) EMU_GS(2) EMU_GS(3) EMU_GS(4) EMU_GS(5) EMU_GS(6)
        EMU_GS(7) EMU_GS(8) EMU_GS(9) EMU_GS(10) EMU_GS(11) EMU_GS(12)
#undef EMU_GS
        default: return cudaErrorInvalidValue;
      }
    }
    if (cudaEventRecord(gs->fork[s], st) != cudaSuccess) return cudaErrorUnknown;
    for (size_t i = 0; i < pl.subs.size(); ++i) {
      if (pl.subs[i].stage != s) continue;
      if (cudaStreamWaitEvent(gs->side[i], gs->fork[s], 0) != cudaSuccess) return cudaErrorUnknown;
      cudaError_t e = launch_sub(pl, pl.subs[i], status, gs->side[i], false);
      if (e != cudaSuccess) return e;
      if (cudaEventRecord(gs->join[i], gs->side[i]) != cudaSuccess) return cudaErrorUnknown;
    }
  }
  for (size_t i = 0; i < pl.subs.size(); ++i)
    if (cudaStreamWaitEvent(st, gs->join[i], 0) != cudaSuccess) return cudaErrorUnknown;
  return cudaGetLastError();
}

static size_t al256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

// Tiles of the products lo .. hi-1 in configuration `cfg`,
// longest-processing-time assigned to `grid` CTA slots (cost = K chunks):
// flat list + CTA offsets.
void lpt_tiles(int lo, int hi, const emu_gemm_desc_t* d, const std::vector<int>& pcfg, int cfg, int grid_max,
               std::vector<int4>* flat, std::vector<int>* cta, int* grid_out) {
  const int BM = kCfgBM[cfg], BN = kCfgBN[cfg];
  std::vector<int4> tiles;
  for (int i = lo; i < hi; ++i) {
    if (pcfg[i] != cfg) continue;
    int tm = static_cast<int>((d[i].m + BM - 1) / BM), tn = static_cast<int>((d[i].n + BN - 1) / BN);
    for (int a = 0; a < tm; ++a)
      for (int b = 0; b < tn; ++b) tiles.push_back(make_int4(i, a, b, 0));
  }
  std::stable_sort(tiles.begin(), tiles.end(), [&](const int4& x, const int4& y) { return d[x.x].k > d[y.x].k; });
  int grid = grid_max;
  if (static_cast<int>(tiles.size()) < grid) grid = std::max<int>(1, static_cast<int>(tiles.size()));
  std::vector<std::vector<int4>> per(grid);
  using Slot = std::pair<int64_t, int>;
  std::priority_queue<Slot, std::vector<Slot>, std::greater<Slot>> heap;
  for (int g = 0; g < grid; ++g) heap.push({0, g});
  for (const int4& t : tiles) {
    Slot s = heap.top();
    heap.pop();
    per[s.second].push_back(t);
    s.first += (d[t.x].k + 31) / 32;
    heap.push(s);
  }
  flat->clear();
  cta->assign(grid + 1, 0);
  for (int g = 0; g < grid; ++g) {
    (*cta)[g] = static_cast<int>(flat->size());
    flat->insert(flat->end(), per[g].begin(), per[g].end());
  }
  (*cta)[grid] = static_cast<int>(flat->size());
  *grid_out = grid;
}

// Stage order of a batch: products sorted by GEMM work per operand element
// (M N K / ((M + N) K)), cut where the cumulative work reaches the
// kStageEnd fractions (one stage for fewer than 8 products or when
// max_stages is 1; no empty stage).  Returns the permutation and the stage
// sizes (*nstages of them).
std::vector<int> stage_order(int count, const emu_gemm_desc_t* d, int max_stages, int* sizes, int* nstages) {
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  *nstages = 1;
  sizes[0] = count;
  if (count < 8 || max_stages < 2) return order;
  auto dens = [&](int i) { return static_cast<double>(d[i].m) * d[i].n / static_cast<double>(d[i].m + d[i].n); };
  auto work = [&](int i) { return static_cast<double>(d[i].m) * d[i].n * d[i].k; };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return dens(a) > dens(b); });
  double total = 0.0;
  for (int i = 0; i < count; ++i) total += work(i);
  double acc = 0.0;
  int n = 0, ns = 0, start = 0;
  for (int s = 0; s < kMaxStages - 1; ++s) {
    while (n < count - 1 && acc < kStageEnd[s] * total) acc += work(order[n++]);
    if (n > start) {
      sizes[ns++] = n - start;
      start = n;
    }
  }
  sizes[ns++] = count - start;
  *nstages = ns;
  return order;
}

// Build a plan: device tables, workspace, tensor maps, LPT tile lists.
emu_status_t build_plan(emu_handle_s* h, int count, const emu_gemm_desc_t* d_in, int p,
                        const std::vector<int>& pcfg_in, int stages, GroupPlan** out) {
  auto* pl = new GroupPlan();
  pl->descs.assign(d_in, d_in + count);
  pl->pcfg = pcfg_in;
  pl->p = p;
  pl->count = count;
  pl->max_stages = stages;
  // the problem table in stage order
  int sizes[kMaxStages] = {};
  const std::vector<int> order = stage_order(count, d_in, stages, sizes, &pl->nstages);
  std::vector<emu_gemm_desc_t> dv(count);
  std::vector<int> pcfg(count);
  for (int i = 0; i < count; ++i) {
    dv[i] = d_in[order[i]];
    pcfg[i] = pcfg_in[order[i]];
  }
  const emu_gemm_desc_t* d = dv.data();
  for (int s = 0, first = 0; s < pl->nstages; first += sizes[s++]) {
    pl->stages[s].first = first;
    pl->stages[s].count = sizes[s];
  }

  std::vector<GProb> probs(count);
  size_t off = 0;
  size_t o_probs = off; off += al256(sizeof(GProb) * count);
  size_t o_maps = off; off += al256(sizeof(CUtensorMap) * 2 * count);
  // one tile list per stage and configuration in use
  std::vector<std::vector<int4>> flats;
  std::vector<std::vector<int>> ctas;
  std::vector<size_t> o_tiles, o_cta;
  for (int s = 0; s < pl->nstages; ++s) {
    const int lo = pl->stages[s].first, hi = lo + pl->stages[s].count;
    for (int cfg = 0; cfg < kNumCfg; ++cfg) {
      if (std::find(pcfg.begin() + lo, pcfg.begin() + hi, cfg) == pcfg.begin() + hi) continue;
      SubPlan sp;
      sp.cfg = cfg;
      sp.stage = s;
      std::vector<int4> flat;
      std::vector<int> cta;
      lpt_tiles(lo, hi, d, pcfg, cfg, h->num_sms * occupancy_of(cfg), &flat, &cta, &sp.grid);
      o_tiles.push_back(off);
      off += al256(sizeof(int4) * std::max<size_t>(flat.size(), 1));
      o_cta.push_back(off);
      off += al256(sizeof(int) * cta.size());
      flats.push_back(std::move(flat));
      ctas.push_back(std::move(cta));
      pl->subs.push_back(sp);
    }
  }
  // block prefix arrays, per stage: [sA | sB | pA | pB], each count_s + 1 long
  std::vector<int> st4;
  std::vector<size_t> st4_off(pl->nstages);
  for (int s = 0; s < pl->nstages; ++s) {
    StagePlan& sg = pl->stages[s];
    const int c = sg.count;
    std::vector<int> sA(c + 1, 0), sB(c + 1, 0), pA(c + 1, 0), pB(c + 1, 0);
    for (int j = 0; j < c; ++j) {
      const emu_gemm_desc_t& dj = d[sg.first + j];
      int64_t M = dj.m, N = dj.n, K = dj.k;
      int64_t rows_a = split_rows(M), rows_b = split_rows(N), nch = (K + 31) / 32;
      sA[j + 1] = sA[j] + static_cast<int>(((M + 7) / 8) * ((K + 2047) / 2048));
      sB[j + 1] = sB[j] + static_cast<int>(((N + 31) / 32) * ((K + 255) / 256));
      pA[j + 1] = pA[j] + static_cast<int>((rows_a * ((nch + 3) / 4) + 7) / 8);
      pB[j + 1] = pB[j] + static_cast<int>((rows_b / 32) * ((nch + 3) / 4));
    }
    sg.scan_blocks = sA[c] + sB[c];
    sg.split_blocks = pA[c] + pB[c];
    st4_off[s] = st4.size();
    st4.insert(st4.end(), sA.begin(), sA.end());
    st4.insert(st4.end(), sB.begin(), sB.end());
    st4.insert(st4.end(), pA.begin(), pA.end());
    st4.insert(st4.end(), pB.begin(), pB.end());
  }
  size_t o_starts = off; off += al256(sizeof(int) * st4.size());
  // per-problem workspace
  size_t o_max = off;
  size_t max_bytes = 0;
  for (int i = 0; i < count; ++i) max_bytes += al256(8 * std::max<int64_t>(d[i].m, 1)) + al256(8 * std::max<int64_t>(d[i].n, 1));
  off += max_bytes;
  std::vector<size_t> o_ws(count);
  for (int i = 0; i < count; ++i) {
    Plan w = plan_I(d[i].m, d[i].n, d[i].k, p);
    o_ws[i] = off;
    off += al256(w.bytes);
  }
  pl->dev_bytes = off;
  if (cudaMalloc(&pl->dev, off) != cudaSuccess) {
    cudaGetLastError();
    delete pl;
    return EMU_ERR_ALLOC;
  }
  uint8_t* base = static_cast<uint8_t*>(pl->dev);
  pl->d_probs = reinterpret_cast<GProb*>(base + o_probs);
  pl->d_maps = reinterpret_cast<CUtensorMap*>(base + o_maps);
  for (size_t i = 0; i < pl->subs.size(); ++i) {
    pl->subs[i].d_tiles = reinterpret_cast<int4*>(base + o_tiles[i]);
    pl->subs[i].d_cta = reinterpret_cast<int*>(base + o_cta[i]);
  }
  int* starts = reinterpret_cast<int*>(base + o_starts);
  for (int s = 0; s < pl->nstages; ++s) {
    StagePlan& sg = pl->stages[s];
    int* st = starts + st4_off[s];
    sg.d_startA_scan = st;
    sg.d_startB_scan = st + (sg.count + 1);
    sg.d_startA_split = st + 2 * (sg.count + 1);
    sg.d_startB_split = st + 3 * (sg.count + 1);
  }
  pl->d_max = reinterpret_cast<unsigned long long*>(base + o_max);
  pl->max_bytes = max_bytes;
  std::vector<CUtensorMap> maps(2 * count);
  size_t moff = 0;
  for (int i = 0; i < count; ++i) {
    GProb& g = probs[i];
    g.A = d[i].A;
    g.B = d[i].B;
    g.C = d[i].C;
    g.lda = d[i].lda;
    g.ldb = d[i].ldb;
    g.ldc = d[i].ldc;
    g.M = static_cast<int>(d[i].m);
    g.N = static_cast<int>(d[i].n);
    g.K = static_cast<int>(d[i].k);
    g.nk32 = static_cast<int>((d[i].k + 31) / 32);
    g.alpha = d[i].alpha;
    g.beta = d[i].beta;
    g.maxA = reinterpret_cast<unsigned long long*>(base + o_max + moff);
    moff += al256(8 * std::max<int64_t>(d[i].m, 1));
    g.maxB = reinterpret_cast<unsigned long long*>(base + o_max + moff);
    moff += al256(8 * std::max<int64_t>(d[i].n, 1));
    Plan w = plan_I(d[i].m, d[i].n, d[i].k, p);
    uint8_t* ws = base + o_ws[i];
    g.EA = reinterpret_cast<int32_t*>(ws + w.off_EA);
    g.FB = reinterpret_cast<int32_t*>(ws + w.off_FB);
    g.hatA = reinterpret_cast<int8_t*>(ws + w.off_hatA);
    g.hatB = reinterpret_cast<int8_t*>(ws + w.off_hatB);
    g.rows_a = w.rows_a;
    g.rows_b = w.rows_b;
    g.nchunks = (d[i].k + 31) / 32;
    // TMA boxes of this product's tile configuration
    const int BM = kCfgBM[pcfg[i]], BN = kCfgBN[pcfg[i]];
    if (!make_tmap_i8(&maps[2 * i], g.hatA, static_cast<uint64_t>(w.cols), static_cast<uint64_t>(w.rows_a), BM) ||
        !make_tmap_i8(&maps[2 * i + 1], g.hatB, static_cast<uint64_t>(w.cols), static_cast<uint64_t>(w.rows_b), BN)) {
      free_plan(pl);
      return EMU_ERR_CUDA;
    }
  }
  bool ok = cudaMemcpy(pl->d_probs, probs.data(), sizeof(GProb) * count, cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(pl->d_maps, maps.data(), sizeof(CUtensorMap) * 2 * count, cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(starts, st4.data(), sizeof(int) * st4.size(), cudaMemcpyHostToDevice) == cudaSuccess;
  for (size_t i = 0; ok && i < pl->subs.size(); ++i)
    ok = (flats[i].empty() || cudaMemcpy(pl->subs[i].d_tiles, flats[i].data(), sizeof(int4) * flats[i].size(),
                                         cudaMemcpyHostToDevice) == cudaSuccess) &&
         cudaMemcpy(pl->subs[i].d_cta, ctas[i].data(), sizeof(int) * ctas[i].size(), cudaMemcpyHostToDevice) ==
             cudaSuccess;
  if (!ok) {
    free_plan(pl);
    return EMU_ERR_CUDA;
  }
  *out = pl;
  return EMU_OK;
}

// Capture the plan's launch sequence into a graph (on a private stream, with
// private side streams for the parallel GEMM branches).
emu_status_t capture_plan(emu_handle_s* h, GroupState* gs, GroupPlan* pl) {
  if (!gs->capture && cudaStreamCreateWithFlags(&gs->capture, cudaStreamNonBlocking) != cudaSuccess)
    return EMU_ERR_CUDA;
  if (!gs->fork[0]) {
    for (int s = 0; s < kMaxStages; ++s)
      if (cudaEventCreateWithFlags(&gs->fork[s], cudaEventDisableTiming) != cudaSuccess) return EMU_ERR_CUDA;
    for (int i = 0; i < kMaxSubs; ++i)
      if (cudaStreamCreateWithFlags(&gs->side[i], cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&gs->join[i], cudaEventDisableTiming) != cudaSuccess)
        return EMU_ERR_CUDA;
  }
  if (prepare_attrs(*pl) != cudaSuccess) return EMU_ERR_CUDA;
  if (cudaStreamBeginCapture(gs->capture, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return EMU_ERR_CUDA;
  cudaError_t le = launch_group(*pl, gs, h->status, gs->capture);
  cudaError_t ce = cudaStreamEndCapture(gs->capture, &pl->graph);
  if (le != cudaSuccess || ce != cudaSuccess) {
    cudaGetLastError();
    return EMU_ERR_CUDA;
  }
  if (cudaGraphInstantiate(&pl->exec, pl->graph, 0) != cudaSuccess) return EMU_ERR_CUDA;
  return EMU_OK;
}

emu_status_t validate(emu_handle_s* h, int count, const emu_gemm_desc_t* d, int p) {
  if (!h || count < 0 || (count > 0 && !d)) return EMU_ERR_INVALID_ARG;
  if (p < EMU_P_MIN || p > EMU_P_MAX) return EMU_ERR_UNSUPPORTED;
  for (int i = 0; i < count; ++i) {
    if (d[i].m < 1 || d[i].n < 1 || d[i].k < 1) return EMU_ERR_INVALID_ARG;
    if (d[i].m > (1 << 24) || d[i].n > (1 << 24) || d[i].k > (1 << 24)) return EMU_ERR_UNSUPPORTED;
    if (!d[i].A || !d[i].B || !d[i].C) return EMU_ERR_INVALID_ARG;
    if (!check_lds(EMU_ROW_MAJOR, d[i].m, d[i].n, d[i].k, d[i].lda, d[i].ldb, d[i].ldc)) return EMU_ERR_INVALID_ARG;
  }
  return EMU_OK;
}

// Run (building and capturing if the product list or the configurations
// changed) with a tile configuration per product.
emu_status_t run_group(emu_handle_s* h, int count, const emu_gemm_desc_t* d, int p, const std::vector<int>& pcfg,
                       int stages, cudaStream_t st) {
  GroupState* gs = state_of(h);
  GroupPlan* pl = gs->plan;
  if (!same_plan(pl, d, count, p, pcfg, stages)) {
    if (pl) {
      cudaDeviceSynchronize();
      free_plan(pl);
      gs->plan = nullptr;
    }
    emu_status_t s = build_plan(h, count, d, p, pcfg, stages, &pl);
    if (s != EMU_OK) return s;
    s = capture_plan(h, gs, pl);
    if (s != EMU_OK) {
      free_plan(pl);
      return s;
    }
    gs->plan = pl;
  }
  trace_begin(h, PH_GEMM, st);
  cudaError_t e = cudaGraphLaunch(pl->exec, st);
  trace_end(h, PH_GEMM, st, 1 + 2 * pl->nstages + static_cast<int>(pl->subs.size()));
  return e == cudaSuccess ? EMU_OK : EMU_ERR_CUDA;
}

// Mean time of `reps` graph replays after a warm-up (ms).
emu_status_t time_group(emu_handle_s* h, int count, const emu_gemm_desc_t* d, int p, const std::vector<int>& pcfg,
                        int stages, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, int reps, float* ms) {
  emu_status_t s = run_group(h, count, d, p, pcfg, stages, st);  // builds, captures and warms up
  if (s != EMU_OK) return s;
  run_group(h, count, d, p, pcfg, stages, st);
  cudaEventRecord(e0, st);
  for (int r = 0; r < reps; ++r) run_group(h, count, d, p, pcfg, stages, st);
  cudaEventRecord(e1, st);
  if (cudaEventSynchronize(e1) != cudaSuccess) return EMU_ERR_CUDA;
  cudaEventElapsedTime(ms, e0, e1);
  *ms /= static_cast<float>(reps);
  return EMU_OK;
}

// Tuning, all timed with CUDA events over graph replays, done once with
// the batch cut into stages (kMaxStages) and once as a single stage; the
// faster outcome is kept, with its stage setting.  For each setting:
// (1) The whole batch in each single configuration (and in the current
// choices): the fastest is the starting point.  (2) Each bucket's products
// alone in every configuration: the fastest is the bucket's candidate (a
// bucket holds a few percent of a mixed batch, so its gain is timed on its
// own products, where it is not lost in the noise of the whole batch).
// (3) The whole batch with every candidate; if that beats the starting
// point it is kept, else each bucket whose choice differs from the
// candidate's is tried on the whole batch and switched if the batch gets at
// least 0.5 % faster.  The buckets' kernels share the GPU (parallel graph
// branches, stages), which is why every decision is confirmed on the whole
// batch.
emu_status_t tune_setting(emu_handle_s* h, int count, const emu_gemm_desc_t* d, int p, int stages,
                          const std::map<std::string, std::vector<int>>& members, cudaStream_t st, cudaEvent_t e0,
                          cudaEvent_t e1, std::vector<int>* out, float* out_ms, int* n_timed) {
  constexpr int kReps = 5;
  GroupState* gs = state_of(h);
  // (1) starting point
  std::vector<int> next = configs_of(gs, count, d, p);
  float base = 0.f;
  emu_status_t s = time_group(h, count, d, p, next, stages, st, e0, e1, kReps, &base);
  ++*n_timed;
  for (int c = 0; s == EMU_OK && c < kNumCfg; ++c) {
    const std::vector<int> uni(count, c);
    if (uni == next) continue;
    float ms = 0.f;
    s = time_group(h, count, d, p, uni, stages, st, e0, e1, kReps, &ms);
    ++*n_timed;
    if (s == EMU_OK && ms < base) {
      base = ms;
      next = uni;
    }
  }
  // (2) per-bucket candidates
  std::map<std::string, int> cand;
  for (auto it = members.begin(); s == EMU_OK && it != members.end(); ++it) {
    std::vector<emu_gemm_desc_t> sub;
    for (int i : it->second) sub.push_back(d[i]);
    const int nsub = static_cast<int>(sub.size());
    float best = 0.f;
    int keep = 0;
    for (int c = 0; s == EMU_OK && c < kNumCfg; ++c) {
      float ms = 0.f;
      s = time_group(h, nsub, sub.data(), p, std::vector<int>(nsub, c), stages, st, e0, e1, kReps, &ms);
      ++*n_timed;
      if (c == 0 || ms < best) {
        best = ms;
        keep = c;
      }
    }
    cand[it->first] = keep;
  }
  // (3) candidates on the whole batch
  std::vector<int> mix(count);
  for (int i = 0; i < count; ++i) mix[i] = cand[bucket_of(d[i], p)];
  if (s == EMU_OK && mix != next) {
    float ms = 0.f;
    s = time_group(h, count, d, p, mix, stages, st, e0, e1, kReps, &ms);
    ++*n_timed;
    if (s == EMU_OK && ms < base) {
      base = ms;
      next = mix;
    } else {
      for (auto it = members.begin(); s == EMU_OK && it != members.end(); ++it) {
        const int c = cand[it->first];
        if (c == next[it->second[0]]) continue;
        std::vector<int> trial = next;
        for (int i : it->second) trial[i] = c;
        s = time_group(h, count, d, p, trial, stages, st, e0, e1, kReps, &ms);
        ++*n_timed;
        if (s == EMU_OK && ms < 0.995f * base) {
          base = ms;
          next = trial;
        }
      }
    }
  }
  *out = next;
  *out_ms = base;
  return s;
}

}  // namespace

void grouped_release(emu_handle_s* h) {
  if (!h->grouped) return;
  auto* gs = static_cast<GroupState*>(h->grouped);
  free_plan(gs->plan);
  if (gs->capture) cudaStreamDestroy(gs->capture);
  for (int i = 0; i < kMaxSubs; ++i) {
    if (gs->side[i]) cudaStreamDestroy(gs->side[i]);
    if (gs->join[i]) cudaEventDestroy(gs->join[i]);
  }
  for (int s = 0; s < kMaxStages; ++s)
    if (gs->fork[s]) cudaEventDestroy(gs->fork[s]);
  delete gs;
  h->grouped = nullptr;
}

}  // namespace emu

using namespace emu;

extern "C" {

emu_status_t emu_dgemm_grouped(emu_handle_t h, int count, const emu_gemm_desc_t* descs, int p, emu_stream_t stream) {
  emu_status_t s = validate(h, count, descs, p);
  if (s != EMU_OK || count == 0) return s;
  cudaSetDevice(h->device);
  GroupState* gs = state_of(h);
  return run_group(h, count, descs, p, configs_of(gs, count, descs, p), stages_of(gs, p),
                   static_cast<cudaStream_t>(stream));
}

emu_status_t emu_dgemm_grouped_loop(emu_handle_t h, int count, const emu_gemm_desc_t* d, int p, emu_stream_t stream) {
  emu_status_t s = validate(h, count, d, p);
  if (s != EMU_OK) return s;
  for (int i = 0; i < count; ++i) {
    s = emu_dgemm(h, EMU_ROW_MAJOR, d[i].m, d[i].n, d[i].k, d[i].alpha, d[i].A, d[i].lda, d[i].B, d[i].ldb,
                  d[i].beta, d[i].C, d[i].ldc, EMU_SCHEME_I, p, stream);
    if (s != EMU_OK) return s;
  }
  return EMU_OK;
}

emu_status_t emu_tune_grouped(emu_handle_t h, int count, const emu_gemm_desc_t* d, int p, const char* path,
                              int* timed, emu_stream_t stream) {
  emu_status_t s = validate(h, count, d, p);
  if (s != EMU_OK || count == 0) return s;
  cudaSetDevice(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  GroupState* gs = state_of(h);
  std::map<std::string, std::vector<int>> members;
  for (int i = 0; i < count; ++i) members[bucket_of(d[i], p)].push_back(i);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int n_timed = 0;
  std::vector<int> next, single;
  float ms_staged = 0.f, ms_single = 0.f;
  s = tune_setting(h, count, d, p, kMaxStages, members, st, e0, e1, &next, &ms_staged, &n_timed);
  if (s == EMU_OK) s = tune_setting(h, count, d, p, 1, members, st, e0, e1, &single, &ms_single, &n_timed);
  int stages = kMaxStages;
  if (s == EMU_OK && ms_single < ms_staged) {
    next = single;
    stages = 1;
  }
  if (s == EMU_OK) gs->tuned[stages_key(p)] = stages;
  if (s == EMU_OK)
    for (auto& kv : members) gs->tuned[kv.first] = next[kv.second[0]];
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != EMU_OK) return s;
  if (timed) *timed = n_timed;
  if (path) {
    std::ofstream f(path);
    if (!f) return EMU_ERR_INVALID_ARG;
    f << "{\n";
    size_t i = 0;
    for (auto& kv : gs->tuned)
      f << "  \"" << kv.first << "\": " << kv.second << (++i < gs->tuned.size() ? ",\n" : "\n");
    f << "}\n";
  }
  return EMU_OK;
}

emu_status_t emu_load_tuning(emu_handle_t h, const char* path) {
  if (!h || !path) return EMU_ERR_INVALID_ARG;
  std::ifstream f(path);
  if (!f) return EMU_ERR_INVALID_ARG;
  GroupState* gs = state_of(h);
  std::string line;
  while (std::getline(f, line)) {
    size_t q1 = line.find('"'), q2 = line.find('"', q1 + 1), c = line.find(':', q2 + 1);
    if (q1 == std::string::npos || q2 == std::string::npos || c == std::string::npos) continue;
    int v = std::atoi(line.c_str() + c + 1);
    const std::string key = line.substr(q1 + 1, q2 - q1 - 1);
    const bool stages = key.size() > 7 && key.compare(key.size() - 7, 7, "_stages") == 0;
    if (stages ? (v < 1 || v > kMaxStages) : (v < 0 || v >= kNumCfg)) return EMU_ERR_INVALID_ARG;
    gs->tuned[key] = v;
  }
  return EMU_OK;
}

}  // extern "C"
