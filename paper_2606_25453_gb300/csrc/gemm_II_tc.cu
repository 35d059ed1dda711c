// gemm_II_tc.cu -- Scheme II on the bf16 tensor cores (tcgen05.mma
// kind::f16) with accumulators in tensor memory, and the CRT.
//
// On sm_103a the 8-bit integer MMA exists only as the warp-level mma.sync.
// The symmetric residues of Eq. (5) (|r| <= 128) are exact bf16 values, the
// products of two of them (|r_a r_b| <= 2^14) are exact, and an FP32 sum of
// up to 960 such products stays an exact integer (|sum| <= 960 * 2^14 <
// 2^24).  So every per-modulus product of Eq. (6) runs as a bf16 GEMM on the
// 5th-generation tensor cores in K segments of 960, and the result is
// bit-identical to the INT8 kernel's.
//
// The work is modulus-major, as in the paper's Scheme II kernel (Sec. IV):
// a persistent kernel walks (modulus, tile) items in that order, so that all
// CTAs work on the same pair of residue planes at the same time and the
// operand tiles are reused from L2 as in one plain GEMM (walking all moduli
// of one tile before the next keeps 16 x more operand data live and reads
// the planes from DRAM about 20 times).  Each item's product stays in TMEM;
// the epilogue reduces it modulo m_l (Eq. 7) and writes only the residue
// bytes (one per output and modulus).  A second kernel then forms the CRT
// sum of Eq. (8) from the residues, reduces it modulo P, lifts it to the
// symmetric range, rounds it once to binary64, scales it back and applies
// the BLAS update (3M combination of Eq. (16) for complex input).
//
// GEMM tile, PAIR form: 256 rows x 256 columns on a pair of CTAs
// (a cluster of two on neighbouring SMs) with tcgen05.mma.cta_group::2: one
// 256 x 256 x 16 MMA per K-step, issued by the even CTA, reads the 128 rows
// of A that each CTA holds and the 256 columns of B of which each CTA holds
// half, and leaves rows 0-127 of the product in the even CTA's TMEM and
// rows 128-255 in the odd one's.  Each CTA's TMA fills only its own shared
// memory (its A rows and its half of B) and counts the bytes on the even
// CTA's stage barrier; the MMA commits release the stage in both CTAs.  Per
// K-step an SM then reads 8 KB of operands from shared memory and receives
// 8 KB by TMA, against 12 + 12 KB for a 128 x 256 tile on one CTA, whose
// shared-memory traffic (192 B per clock at full tensor rate against 128 B
// per clock of bandwidth) caps it near two thirds of the tensor peak; the
// smaller stages also fit six deep instead of four.  Measured on GB300 the
// pair form is nevertheless not faster than the single-CTA form (128 x 256
// tile, tcgen05.mma.cta_group::1), which is the default; the pair form runs
// with EMU_II_CLUSTER=2.
//
// Two FP32 accumulators take all 512 TMEM columns of each CTA and alternate
// between K segments, so the MMAs of one segment overlap the reduction of
// the last.  Roles (320 threads per CTA): warps 0-7 drain (warp w: TMEM
// lanes = tile rows 32 (w % 4) .., columns 128 (w / 4) .. +127; each
// finished segment is added to a running residue, four per register, with
// FP32 arithmetic only), warp 8 lane 0 TMA, warp 9 TMEM allocation and
// (lane 0 of the even CTA) MMAs.
// All waits are bounded; a timeout sets the status word, raises the abort
// flag of both CTAs of a pair for the other roles, and the TMEM is still
// released.
#include <cstdlib>
#include <type_traits>

#include "crt_core.cuh"
#include "emu_internal.h"
#include "tc_core.cuh"

namespace emu {
namespace {

constexpr int kBM = 128, kBN = 256;  // accumulator tile of one CTA: TMEM lanes x FP32 columns
constexpr int kThreads = 320;
constexpr int kDrainWarps = 8;
constexpr int kProducerWarp = 8, kMmaWarp = 9;
constexpr uint32_t kTmemCols = 512;
constexpr int kSegStages = 15;  // 64-wide K chunks per exact FP32 segment (960 * 2^14 < 2^24)
static_assert(kSegStages * 64 * 16384 < (1 << 24), "segment sums must stay exact in FP32");

template <bool PAIR>
struct CfgII {
  static constexpr int kRowsB = PAIR ? kBN / 2 : kBN;  // B rows (output columns) this CTA loads
  static constexpr int kBlkA = kBM * 128;               // one K chunk: 128 rows x 64 bf16, 128-byte rows
  static constexpr int kBlkB = kRowsB * 128;
  static constexpr int kStageBytes = kBlkA + kBlkB;
  static constexpr int kStages = PAIR ? 6 : 4;
  static constexpr int kSmem = kStages * kStageBytes + 1024 + 256;
  static_assert(kSmem <= 232448, "shared memory");
  static_assert(kStageBytes % 1024 == 0, "stages keep the 1024-byte swizzle alignment");
};

struct KParamsIITC {
  CUtensorMap tA;  // bf16 planes as bytes: 128-byte x 128-row boxes, 128-byte swizzle
  CUtensorMap tB;  // 128-byte x (256 or 128)-row boxes
  int nst;         // 64-wide K chunks per plane
  int tiles_m;     // 128-row tiles of the residue matrices (even with CTA pairs)
  int tiles_mu;    // row units of the work list: 256-row pair tiles or 128-row tiles
  int tiles_n;     // 256-column tiles
  int nplanes;     // NSET * nm residue planes (plane p = set * nm + l)
  int nm;
  int rowsA_pad, rowsB_pad;
  uint8_t* R;      // residues: plane p, row r, column c at R[(p * tiles_m * 128 + r) * ldr + c]
  int64_t ldr;     // tiles_n * 256
  int* status;
};

// Instruction descriptor: bf16 x bf16 -> F32, both K-major, M x N.
__device__ __forceinline__ uint32_t idesc_bf16(int M, int N) {
  return (1u << 4)                                  // D format F32
         | (1u << 7) | (1u << 10)                   // A, B format BF16
         | (static_cast<uint32_t>(N >> 3) << 17)    // N / 8
         | (static_cast<uint32_t>(M >> 4) << 24);   // M / 16
}

template <bool PAIR>
__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  if constexpr (PAIR)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
  else
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive on the barrier at shared::cluster address `bar` (this CTA's or the
// peer's) once every MMA issued so far by this thread has completed.
__device__ __forceinline__ void umma_commit_pair(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

template <bool PAIR>
__device__ __forceinline__ void tmem_alloc_all(uint32_t* slot) {
  if constexpr (PAIR) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  } else {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
}

template <bool PAIR>
__device__ __forceinline__ void tmem_free_all(uint32_t tmem) {
  if constexpr (PAIR)
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  else
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// shared::cluster address of the object at shared::cta address `saddr` in
// the CTA of the cluster with rank `rank`.
__device__ __forceinline__ uint32_t cluster_addr(uint32_t saddr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
  return r;
}

// 2D tiled TMA load into this CTA's shared memory, completion counted on the
// barrier at shared::cluster address `bar`, which may be the peer CTA's.
__device__ __forceinline__ void tma_load_2d_pair(void* smem_dst, const void* desc, uint32_t bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(smem_dst)),
      "l"(reinterpret_cast<uint64_t>(desc)), "r"(bar), "r"(x), "r"(y)
      : "memory");
}

// Arrive (release, cluster scope) on the barrier at shared::cluster address `bar`.
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t bar) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait_acq_cluster(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Abort flags: this CTA's, and (pairs) the shared::cluster address of the
// peer's, so that a role that gives up stops both CTAs of the pair.
struct AbortFlag {
  volatile int* local;
  uint32_t peer;  // 0: no peer
};

__device__ __forceinline__ void raise_abort(const AbortFlag& ab) {
  *ab.local = 1;
  if (ab.peer) asm volatile("st.relaxed.cluster.shared::cluster.u32 [%0], %1;" ::"r"(ab.peer), "r"(1u) : "memory");
}

// Bounded wait unless the pair already gave up; false means "stop".  With
// `cluster_acq` the wait acquires at cluster scope (arrivals from the peer).
__device__ __forceinline__ bool wait_pair(uint64_t* bar, uint32_t parity, const AbortFlag& ab, int* status,
                                          bool cluster_acq = false) {
  // fast path: the phase is already complete (no abort-flag load on the way)
  if (cluster_acq ? mbar_try_wait_acq_cluster(bar, parity) : mbar_try_wait(bar, parity)) return true;
  if (*ab.local) return false;
  if (cluster_acq) {
    const long long t0 = clock64();
    while (!mbar_try_wait_acq_cluster(bar, parity)) {
      if (*ab.local) return false;
      if (clock64() - t0 > kWaitCycles) {
        set_status(status, ST_TIMEOUT);
        raise_abort(ab);
        return false;
      }
    }
    return true;
  }
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (*ab.local) return false;
    if (clock64() - t0 > kWaitCycles) {
      set_status(status, ST_TIMEOUT);
      raise_abort(ab);
      return false;
    }
  }
  return true;
}

// 16 consecutive 32-bit TMEM columns of this thread's lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

// A multiple of m_l added to (or removed from) an exact int32 sum, keeping
// its residue: x = hi 2^16 + lo -> hi (2^16 mod m) + lo, |result| < 2^22.1
// (p16: the symmetric residue of 2^16 mod m, |p16| <= 128).
__device__ __forceinline__ int fold16(int x, int p16) { return (x >> 16) * p16 + (x & 0xFFFF); }

// x mod m in [0, m) for |x| < 2^23: the quotient estimate floor(RN(x) *
// RN(1/m)) errs by at most one (|x / m| < 2^16, relative error < 2^-22),
// and one correction each way finishes.
__device__ __forceinline__ int mod_small(int x, int m, float inv) {
  const int q = __float2int_rd(__fmul_rn(__int2float_rn(x), inv));
  int r = x - q * m;
  if (r < 0) r += m;
  if (r >= m) r -= m;
  return r;
}

__device__ __forceinline__ void tile_coords(int tile, int tiles_m, int tiles_n, int& tm, int& tn) {
  constexpr int G = 16;  // row tiles per group of the tile order (16: 1-2 % faster than 8 at n = 8192-16384)
  int per_group = G * tiles_n;
  int g = tile / per_group;
  int first = g * G;
  int gsz = tiles_m - first < G ? tiles_m - first : G;
  int in = tile - g * per_group;
  tm = first + in % gsz;
  tn = in / gsz;
}

// Work item i: plane p = i / (tiles per plane), then the tile; tm is this
// CTA's 128-row tile (a pair's rows 0-127 on the even CTA, 128-255 on the
// odd one).
template <bool PAIR>
__device__ __forceinline__ void item_coords(const KParamsIITC& kp, int item, int crank, int& p, int& tm, int& tn) {
  const int per_plane = kp.tiles_mu * kp.tiles_n;
  p = item / per_plane;
  int tu;
  tile_coords(item - p * per_plane, kp.tiles_mu, kp.tiles_n, tu, tn);
  tm = PAIR ? 2 * tu + crank : tu;
}

template <bool PAIR>
__global__ void __launch_bounds__(kThreads, 1)
    gemm_II_tc_kernel(const __grid_constant__ KParamsIITC kp, const __grid_constant__ ModTables mt) {
  using Cfg = CfgII<PAIR>;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* smem = smem_raw + (base - raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + Cfg::kStages * Cfg::kStageBytes);
  uint64_t* empty = full + Cfg::kStages;
  uint64_t* acc_full = empty + Cfg::kStages;  // two accumulators
  uint64_t* acc_empty = acc_full + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 2);
  volatile int* abort_local = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t crank = PAIR ? cluster_ctarank() : 0u;  // 0: the pair's MMA-issuing CTA
  const bool leader = crank == 0;
  const int cid = PAIR ? static_cast<int>(cluster_id_x()) : static_cast<int>(blockIdx.x);
  const int ncl = PAIR ? static_cast<int>(cluster_count_x()) : static_cast<int>(gridDim.x);
  if (threadIdx.x == 0) {
    for (int s = 0; s < Cfg::kStages; ++s) {
      mbar_init(&full[s], 1);   // the even CTA's expect-tx arrival (+ the bytes of both CTAs)
      mbar_init(&empty[s], 1);  // one MMA commit
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], PAIR ? 2 * kDrainWarps : kDrainWarps);  // one arrival per drain warp
    }
    *abort_local = 0;
    fence_mbar_init();
  }
  if (warp == kMmaWarp) {  // the whole warp allocates the tensor memory (both CTAs of a pair)
    tmem_alloc_all<PAIR>(tmem_slot);
    tc_fence_before();
  }
  // barriers and flags initialised in both CTAs before either touches the peer's
  if (PAIR)
    cluster_sync_all();
  else
    __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  AbortFlag ab;
  ab.local = abort_local;
  ab.peer = PAIR ? cluster_addr(smem_u32(const_cast<int*>(abort_local)), crank ^ 1u) : 0u;

  const int nitems = kp.nplanes * kp.tiles_mu * kp.tiles_n;
  const int my_items = cid < nitems ? (nitems - 1 - cid) / ncl + 1 : 0;
  const int nseg = (kp.nst + kSegStages - 1) / kSegStages;

  if (warp == kProducerWarp) {
    // ---------------------------------------------------------------- producer (both CTAs)
    if (lane == 0) {
      tma_prefetch_desc(&kp.tA);
      tma_prefetch_desc(&kp.tB);
      uint32_t j = 0;
      bool stop = false;
      for (int t = 0; t < my_items && !stop; ++t) {
        int p, tm, tn;
        item_coords<PAIR>(kp, cid + t * ncl, static_cast<int>(crank), p, tm, tn);
        const int ya = p * kp.rowsA_pad + tm * kBM;
        const int yb = p * kp.rowsB_pad + tn * kBN + static_cast<int>(crank) * Cfg::kRowsB;
        for (int ks = 0; ks < kp.nst; ++ks, ++j) {
          const uint32_t stage = j % Cfg::kStages;
          if (j >= static_cast<uint32_t>(Cfg::kStages) &&
              !wait_pair(&empty[stage], ((j / Cfg::kStages) & 1u) ^ 1u, ab, kp.status)) {
            stop = true;
            break;
          }
          uint8_t* sA = smem + stage * Cfg::kStageBytes;
          if (PAIR) {
            // both CTAs' bytes are counted on the even CTA's barrier
            const uint32_t bar = cluster_addr(smem_u32(&full[stage]), 0u);
            if (leader) mbar_arrive_expect_tx(&full[stage], 2 * Cfg::kStageBytes);
            tma_load_2d_pair(sA, &kp.tA, bar, ks * 128, ya);
            tma_load_2d_pair(sA + Cfg::kBlkA, &kp.tB, bar, ks * 128, yb);
          } else {
            mbar_arrive_expect_tx(&full[stage], Cfg::kStageBytes);
            tma_load_2d(sA, &kp.tA, &full[stage], ks * 128, ya);
            tma_load_2d(sA + Cfg::kBlkA, &kp.tB, &full[stage], ks * 128, yb);
          }
        }
      }
      // Drain: wait until the last MMA commits have arrived on this CTA's
      // stage barriers (a pair's odd CTA gets them from the even one), so
      // that none lands after the CTA exits.
      if (!stop && PAIR) {
        for (uint32_t jj = j; jj < j + Cfg::kStages; ++jj) {
          if (jj < static_cast<uint32_t>(Cfg::kStages)) continue;
          const uint32_t stage = jj % Cfg::kStages;
          if (!wait_pair(&empty[stage], ((jj / Cfg::kStages) & 1u) ^ 1u, ab, kp.status)) break;
        }
      }
    }
    __syncwarp();
  } else if (warp == kMmaWarp) {
    // ---------------------------------------------------------------- MMA issuer (even CTA of a pair)
    if (lane == 0 && leader) {
      const uint32_t idesc = idesc_bf16(PAIR ? 2 * kBM : kBM, kBN);
      const uint32_t peer = 1u;
      const uint32_t total = static_cast<uint32_t>(my_items) * static_cast<uint32_t>(kp.nst);
      uint32_t it = 0, seg = 0;
      bool stop = false;
      bool ready = false;  // the probe after the previous stage's MMAs already saw this stage's data
      for (int t = 0; t < my_items && !stop; ++t)
        for (int ks = 0; ks < kp.nst; ++ks, ++it) {
          const bool first = ks % kSegStages == 0;
          const uint32_t b = seg & 1u;
          if (first && seg >= 2) {  // the drain warps must have read this accumulator's last segment
            if (!wait_pair(&acc_empty[b], ((seg >> 1) - 1) & 1u, ab, kp.status, PAIR)) {
              stop = true;
              break;
            }
            tc_fence_after();
          }
          const uint32_t stage = it % Cfg::kStages;
          if (!ready && !wait_pair(&full[stage], (it / Cfg::kStages) & 1u, ab, kp.status)) {
            stop = true;
            break;
          }
          tc_fence_after();
          const uint32_t sA = base + stage * Cfg::kStageBytes;
#pragma unroll
          for (int q = 0; q < 4; ++q)  // four K-steps of 16 inside the 128-byte rows
            umma_bf16<PAIR>(tmem + b * kBN, smem_desc_k128(sA + 32 * q), smem_desc_k128(sA + Cfg::kBlkA + 32 * q),
                            idesc, (first && q == 0) ? 0u : 1u);
          // Probe (without blocking) the next stage's data while these MMAs
          // are queued: when it has arrived, the next MMAs follow at once
          // instead of after a blocking wait, which would let the tensor
          // pipe run dry.
          ready = it + 1 < total &&
                  mbar_test_wait(&full[(it + 1) % Cfg::kStages], ((it + 1) / Cfg::kStages) & 1u);
          // the stage is free (in both CTAs of a pair) once these MMAs finish
          if (PAIR) {
            umma_commit_pair(smem_u32(&empty[stage]));
            umma_commit_pair(cluster_addr(smem_u32(&empty[stage]), peer));
          } else {
            umma_commit(&empty[stage]);
          }
          if ((ks + 1) % kSegStages == 0 || ks + 1 == kp.nst) {
            if (PAIR) {
              umma_commit_pair(smem_u32(&acc_full[b]));
              umma_commit_pair(cluster_addr(smem_u32(&acc_full[b]), peer));
            } else {
              umma_commit(&acc_full[b]);
            }
            ++seg;
          }
        }
    }
    __syncwarp();
  } else {
    // ---------------------------------------------------------------- drain (both CTAs)
    const int hh = warp >> 2;
    const int row_in_tile = (warp & 3) * 32 + lane;
    const uint32_t lane_addr = tmem + (static_cast<uint32_t>((warp & 3) * 32) << 16) + static_cast<uint32_t>(hh * 128);
    // the accumulators are released to the even CTA's MMA thread
    const uint32_t acc_empty0 = PAIR ? cluster_addr(smem_u32(&acc_empty[0]), 0u) : 0u;
    const uint32_t acc_empty1 = PAIR ? cluster_addr(smem_u32(&acc_empty[1]), 0u) : 0u;
    uint32_t seg = 0;
    bool stop = false;
    for (int t = 0; t < my_items && !stop; ++t) {
      int p, tm, tn;
      item_coords<PAIR>(kp, cid + t * ncl, static_cast<int>(crank), p, tm, tn);
      const int l = p % kp.nm;
      const int m = static_cast<int>(mt.mods[l]);
      const int p16 = mt.pow16[l][1];
      const float inv = mt.inv[l];
      // Exact integer sums of this thread's 128 columns over the segments so
      // far: each segment adds one exact FP32 value per output, and only the
      // final sum is reduced mod m -- two instructions per output and
      // segment, because the drain competes for issue slots with the MMA
      // thread, which must keep the tensor pipe fed.
      int run[128];
#pragma unroll
      for (int i = 0; i < 128; ++i) run[i] = 0;
      for (int s = 0; s < nseg; ++s, ++seg) {
        const uint32_t b = seg & 1u;
        // one lane per warp polls the barrier (256 polling threads slowed the
        // other roles), the warp follows it
        bool ok = true;
        if (lane == 0) ok = wait_pair(&acc_full[b], (seg >> 1) & 1u, ab, kp.status);
        ok = __shfl_sync(0xFFFFFFFFu, ok ? 1 : 0, 0) != 0;
        __syncwarp();
        if (!ok) {
          stop = true;
          break;
        }
        tc_fence_after();
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          uint32_t v[16];
          tmem_ld16(lane_addr + b * kBN + 16 * q, v);
          tmem_wait_ld();
          if (q == 7) {  // the MMAs may refill this accumulator now
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
              if (PAIR)
                mbar_arrive_cluster(b ? acc_empty1 : acc_empty0);
              else
                mbar_arrive(&acc_empty[b]);
            }
          }
#pragma unroll
          for (int i = 0; i < 16; ++i) run[16 * q + i] += __float2int_rn(__uint_as_float(v[i]));
        }
        // |segment sum| <= 960 * 2^14 < 2^24: fold every 64 segments so that
        // the int32 sums never overflow, whatever K is
        if ((s & 63) == 63) {
#pragma unroll
          for (int i = 0; i < 128; ++i) run[i] = fold16(run[i], p16);
        }
      }
      if (stop) break;
      // Eq. (7): residues in [0, m), 128 bytes of this thread's row
      uint4* dst = reinterpret_cast<uint4*>(
          kp.R + (static_cast<int64_t>(p) * kp.tiles_m * kBM + tm * kBM + row_in_tile) * kp.ldr + tn * kBN + hh * 128);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        uint32_t wv[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          uint32_t o = 0;
#pragma unroll
          for (int k = 0; k < 4; ++k)
            o |= static_cast<uint32_t>(mod_small(fold16(run[16 * i + 4 * e + k], p16), m, inv)) << (8 * k);
          wv[e] = o;
        }
        dst[i] = make_uint4(wv[0], wv[1], wv[2], wv[3]);
      }
    }
  }
  tc_fence_before();
  // no CTA of a pair leaves while the other may still touch its shared or tensor memory
  if (PAIR)
    cluster_sync_all();
  else
    __syncthreads();
  if (warp == kMmaWarp) {
    tc_fence_after();
    tmem_free_all<PAIR>(tmem);
  }
}

// ---------------------------------------------------------------- CRT
struct KParamsCRT {
  const uint8_t* R;
  int64_t ldr, plane;  // residue row pitch and plane size (bytes)
  int M, N, nm;
  const int32_t* EA;
  const int32_t* FB;
  int escale;
  double alpha_re, alpha_im, beta_re, beta_im;
  void* C;
  int64_t ldc;
  int plain;  // alpha = 1, beta = 0: C = the result (no FP64 update arithmetic)
};

// Output columns per thread of the CRT kernel: four in the real modes (one
// 32-bit word per residue plane; two measured no faster), two in the complex
// ones (three planes per modulus in 16-bit words, so that every residue is
// loaded up front).
constexpr int crt_cols(int mode) { return (mode == II_Z3M || mode == II_C3M) ? 2 : 4; }

// One thread per row and crt_cols consecutive columns: the CRT sums of Eq.
// (8) from the residue planes (3M: Re = T1 - T2, Im = T3 - T1 - T2 mod m,
// Eq. 16), S mod P with the symmetric lift, binary64, scaling and the update.
template <int MODE, int L>
__global__ void __launch_bounds__(256) crt_II_kernel(const __grid_constant__ KParamsCRT kp,
                                                     const __grid_constant__ CrtTables ct,
                                                     const __grid_constant__ ModTables mt) {
  constexpr bool CPLX = MODE == II_Z3M || MODE == II_C3M;
  constexpr int kCols = crt_cols(MODE);
  const int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int ncq = (kp.N + kCols - 1) / kCols;
  if (idx >= static_cast<int64_t>(kp.M) * ncq) return;
  const int row = static_cast<int>(idx / ncq), c0 = static_cast<int>(idx % ncq) * kCols;
  const uint8_t* const p = kp.R + static_cast<int64_t>(row) * kp.ldr + c0;
  const int erow = kp.EA[row] + kp.escale;
  if constexpr (!CPLX) {
    // all residue words first (independent, predicated loads in flight
    // together), then the sums: a load per modulus waited on in turn left
    // the kernel bound by memory latency
    uint32_t wl[kMaxModuli];
#pragma unroll
    for (int l = 0; l < kMaxModuli; ++l) {
      const uint8_t* q = p + static_cast<int64_t>(l) * kp.plane;
      if constexpr (kCols == 4)
        wl[l] = l < kp.nm ? __ldg(reinterpret_cast<const uint32_t*>(q)) : 0u;
      else
        wl[l] = l < kp.nm ? __ldg(reinterpret_cast<const unsigned short*>(q)) : 0u;
    }
    CrtLazy acc[kCols];
#pragma unroll
    for (int c = 0; c < kCols; ++c) crt_lazy_init(acc[c]);
#pragma unroll
    for (int l = 0; l < kMaxModuli; ++l) {
      if (l >= kp.nm) break;
#pragma unroll
      for (int c = 0; c < kCols; ++c) crt_lazy_acc<L>(acc[c], ct, l, (wl[l] >> (8 * c)) & 0xFFu);
    }
#pragma unroll
    for (int c = 0; c < kCols; ++c) {
      const int cidx = c0 + c;
      if (cidx >= kp.N) break;
      const double xr = scale2_fast(crt_finish_lazy(acc[c], ct), erow + kp.FB[cidx]);
      if (kp.plain) {  // FP64 is slow on this GPU: no multiply by alpha = 1
        if (MODE == II_F64)
          static_cast<double*>(kp.C)[static_cast<int64_t>(row) * kp.ldc + cidx] = xr;
        else
          static_cast<float*>(kp.C)[static_cast<int64_t>(row) * kp.ldc + cidx] = static_cast<float>(xr);
      } else if (MODE == II_F64) {
        double* cp = static_cast<double*>(kp.C) + static_cast<int64_t>(row) * kp.ldc + cidx;
        *cp = blas_update(kp.alpha_re, xr, kp.beta_re, kp.beta_re != 0.0 ? *cp : 0.0);
      } else {
        float* cp = static_cast<float*>(kp.C) + static_cast<int64_t>(row) * kp.ldc + cidx;
        *cp = static_cast<float>(
            blas_update(kp.alpha_re, xr, kp.beta_re, kp.beta_re != 0.0 ? static_cast<double>(*cp) : 0.0));
      }
    }
  } else {
    // two columns per thread: all 3 N_m residue pairs (16-bit words) first,
    // then the sums with every table index a compile-time constant
    const int64_t set = static_cast<int64_t>(kp.nm) * kp.plane;
    uint32_t v1[kMaxModuli], v2[kMaxModuli], v3[kMaxModuli];
#pragma unroll
    for (int l = 0; l < kMaxModuli; ++l) {
      const bool on = l < kp.nm;
      const uint8_t* q = p + static_cast<int64_t>(l) * kp.plane;
      v1[l] = on ? __ldg(reinterpret_cast<const unsigned short*>(q)) : 0u;
      v2[l] = on ? __ldg(reinterpret_cast<const unsigned short*>(q + set)) : 0u;
      v3[l] = on ? __ldg(reinterpret_cast<const unsigned short*>(q + 2 * set)) : 0u;
    }
    CrtLazy are[kCols], aim[kCols];
#pragma unroll
    for (int c = 0; c < kCols; ++c) {
      crt_lazy_init(are[c]);
      crt_lazy_init(aim[c]);
    }
#pragma unroll
    for (int l = 0; l < kMaxModuli; ++l) {
      if (l >= kp.nm) break;
      const int m = static_cast<int>(mt.mods[l]);
#pragma unroll
      for (int c = 0; c < kCols; ++c) {
        // T1 - T2 and T3 - T1 - T2 modulo m, kept non-negative by adding m
        // and 2m instead of reducing: w_l m_l is a multiple of P, so the
        // offsets leave S mod P unchanged (residues below 3 m)
        const int t1 = (v1[l] >> (8 * c)) & 0xFF, t2 = (v2[l] >> (8 * c)) & 0xFF, t3 = (v3[l] >> (8 * c)) & 0xFF;
        const int re = t1 - t2 + m;
        const int im = t3 - t1 - t2 + 2 * m;
        crt_lazy_acc<L>(are[c], ct, l, static_cast<uint32_t>(re));
        crt_lazy_acc<L>(aim[c], ct, l, static_cast<uint32_t>(im));
      }
    }
#pragma unroll
    for (int c = 0; c < kCols; ++c) {
      const int cidx = c0 + c;
      if (cidx >= kp.N) break;
      const int sc = erow + kp.FB[cidx];
      const double xr = scale2_fast(crt_finish_lazy(are[c], ct), sc);
      const double xi = scale2_fast(crt_finish_lazy(aim[c], ct), sc);
      // complex update in binary64; complex64 output rounds each part once more
      using TO = typename std::conditional<MODE == II_C3M, float, double>::type;
      TO* cp = static_cast<TO*>(kp.C) + 2 * (static_cast<int64_t>(row) * kp.ldc + cidx);
      if (kp.plain) {
        cp[0] = static_cast<TO>(xr);
        cp[1] = static_cast<TO>(xi);
        continue;
      }
      double tr = __fma_rn(kp.alpha_re, xr, -__dmul_rn(kp.alpha_im, xi));
      double ti = __fma_rn(kp.alpha_re, xi, __dmul_rn(kp.alpha_im, xr));
      if (kp.beta_re != 0.0 || kp.beta_im != 0.0) {
        const double cr = static_cast<double>(cp[0]), ci = static_cast<double>(cp[1]);
        tr = __dadd_rn(tr, __fma_rn(kp.beta_re, cr, -__dmul_rn(kp.beta_im, ci)));
        ti = __dadd_rn(ti, __fma_rn(kp.beta_re, ci, __dmul_rn(kp.beta_im, cr)));
      }
      cp[0] = static_cast<TO>(tr);
      cp[1] = static_cast<TO>(ti);
    }
  }
}

// Largest number of co-resident CTA pairs of the GEMM kernel (0 if it cannot
// run in clusters of two).
int max_pairs() {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(2u * 64u);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = CfgII<true>::kSmem;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, gemm_II_tc_kernel<true>, &cfg) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  return n;
}

template <bool PAIR>
cudaError_t launch_residues_t(const GemmIIArgs& a, int nsets, const ModTables& mt, cudaStream_t st) {
  using Cfg = CfgII<PAIR>;
  cudaError_t e = cudaFuncSetAttribute(gemm_II_tc_kernel<PAIR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       Cfg::kSmem);
  if (e != cudaSuccess) return e;
  KParamsIITC kp;
  kp.tA = *a.descA;
  kp.tB = *a.descB;
  kp.nst = a.nk32 / 2;  // planes are padded to 128 K-elements
  kp.tiles_m = (a.M + kBM - 1) / kBM;
  if (PAIR) kp.tiles_m += kp.tiles_m & 1;  // whole pair tiles: the residue planes hold them
  kp.tiles_mu = PAIR ? kp.tiles_m / 2 : kp.tiles_m;
  kp.tiles_n = (a.N + kBN - 1) / kBN;
  kp.nplanes = nsets * a.nm;
  kp.nm = a.nm;
  kp.rowsA_pad = a.rowsA_pad;
  kp.rowsB_pad = a.rowsB_pad;
  kp.R = a.scratch;
  kp.ldr = static_cast<int64_t>(kp.tiles_n) * kBN;
  kp.status = a.status;
  const int nitems = kp.nplanes * kp.tiles_mu * kp.tiles_n;
  if (nitems == 0 || kp.nst == 0) return cudaSuccess;
  if (!PAIR) {
    const int grid = nitems < a.num_sms ? nitems : a.num_sms;
    gemm_II_tc_kernel<false><<<grid, kThreads, Cfg::kSmem, st>>>(kp, mt);
    return cudaGetLastError();
  }
  static int mc = -1;
  if (mc < 0) mc = max_pairs();
  if (mc <= 0) return cudaErrorInvalidConfiguration;
  const int npairs = nitems < mc ? nitems : mc;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(static_cast<unsigned>(2 * npairs));
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = Cfg::kSmem;
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, gemm_II_tc_kernel<true>, kp, mt);
}

cudaError_t launch_residues(const GemmIIArgs& a, int nsets, const ModTables& mt, cudaStream_t st) {
  if (a.cluster == 2) return launch_residues_t<true>(a, nsets, mt, st);
  if (a.cluster == 1) return launch_residues_t<false>(a, nsets, mt, st);
  return cudaErrorInvalidValue;
}

template <int MODE>
cudaError_t launch_crt(const GemmIIArgs& a, const ModTables& mt, const CrtTables& ct, cudaStream_t st) {
  KParamsCRT kp;
  const int cl = a.cluster;
  const int tiles_m = ((a.M + kBM - 1) / kBM + cl - 1) / cl * cl;
  kp.R = a.scratch;
  kp.ldr = static_cast<int64_t>((a.N + kBN - 1) / kBN) * kBN;
  kp.plane = static_cast<int64_t>(tiles_m) * kBM * kp.ldr;
  kp.M = a.M;
  kp.N = a.N;
  kp.nm = a.nm;
  kp.EA = a.EA;
  kp.FB = a.FB;
  kp.escale = a.escale;
  kp.alpha_re = a.alpha_re;
  kp.alpha_im = a.alpha_im;
  kp.beta_re = a.beta_re;
  kp.beta_im = a.beta_im;
  kp.C = a.C;
  kp.ldc = a.ldc;
  kp.plain = a.alpha_re == 1.0 && a.alpha_im == 0.0 && a.beta_re == 0.0 && a.beta_im == 0.0;
  const int64_t threads = static_cast<int64_t>(a.M) * ((a.N + crt_cols(MODE) - 1) / crt_cols(MODE));
  if (threads == 0) return cudaSuccess;
  // limbs of P: 3 for up to 12 moduli (P < 2^96), 4 up to 16 (P < 2^128), else 5
  const unsigned grid = static_cast<unsigned>((threads + 255) / 256);
  if (ct.P[4] != 0)
    crt_II_kernel<MODE, 5><<<grid, 256, 0, st>>>(kp, ct, mt);
  else if (ct.P[3] != 0)
    crt_II_kernel<MODE, 4><<<grid, 256, 0, st>>>(kp, ct, mt);
  else
    crt_II_kernel<MODE, 3><<<grid, 256, 0, st>>>(kp, ct, mt);
  return cudaGetLastError();
}

// part: 1 = the residue GEMM, 2 = the CRT kernel, 3 = both.
template <int MODE>
cudaError_t launch_mode(const GemmIIArgs& a, const ModTables& mt, const CrtTables& ct, cudaStream_t st, int part) {
  constexpr int NSET = (MODE == II_Z3M || MODE == II_C3M) ? 3 : 1;
  if (part & 1) {
    cudaError_t e = launch_residues(a, NSET, mt, st);
    if (e != cudaSuccess) return e;
  }
  return (part & 2) ? launch_crt<MODE>(a, mt, ct, st) : cudaSuccess;
}

}  // namespace

int gemm_II_tc_tile_m() { return kBM; }
int gemm_II_tc_tile_n() { return kBN; }

size_t gemm_II_tc_residue_bytes(int64_t M, int64_t N, int nm, bool is_complex, int cluster) {
  const int64_t tiles_m = ((M + kBM - 1) / kBM + cluster - 1) / cluster * cluster;
  const int64_t tiles_n = (N + kBN - 1) / kBN;
  return static_cast<size_t>(is_complex ? 3 : 1) * nm * static_cast<size_t>(tiles_m * kBM) *
         static_cast<size_t>(tiles_n * kBN);
}

// CTAs per GEMM tile of the Scheme II tcgen05 kernel: 1 (one CTA on a
// 128 x 256 tile; the default) or 2 (a CTA pair on one 256 x 256 tile,
// tcgen05.mma.cta_group::2) with EMU_II_CLUSTER=2.  The B tensor map's box
// is 256 / cluster rows.
int gemm_II_tc_cluster() {
  static int v = 0;
  if (v == 0) {
    const char* e = std::getenv("EMU_II_CLUSTER");
    v = (e && std::atoi(e) == 2) ? 2 : 1;
  }
  return v;
}

cudaError_t launch_gemm_II_tc(int out_mode, const GemmIIArgs& a, const ModTables& mt, const CrtTables& ct,
                              cudaStream_t st, int part) {
  switch (out_mode) {
    case II_F64:
      return launch_mode<II_F64>(a, mt, ct, st, part);
    case II_F32:
      return launch_mode<II_F32>(a, mt, ct, st, part);
    case II_Z3M:
      return launch_mode<II_Z3M>(a, mt, ct, st, part);
    case II_C3M:
      return launch_mode<II_C3M>(a, mt, ct, st, part);
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace emu
