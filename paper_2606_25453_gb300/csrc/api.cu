// api.cu -- the C ABI (include/emugemm.h): handle, workspace, host-side
// method constants, tensor maps, and the launch sequences of the hot path
// (scan -> split -> fused GEMM) for emu_dgemm / emu_sgemm / emu_zgemm and
// the exported intermediate steps.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "emu_internal.h"
#include "emu_handle.h"
#include "../../include/emugemm.h"

namespace emu {

// ================================================================ constants
// Greedy descending list of pairwise-coprime integers from 256 (Sec. II-C-2
// names 256, 255, 253, ...).
int host_moduli(int nm, int32_t* out) {
  int cnt = 0;
  for (int x = 256; x >= 2 && cnt < nm; --x) {
    bool ok = true;
    for (int j = 0; j < cnt && ok; ++j) {
      int a = x, b = out[j];
      while (b) {
        int t = a % b;
        a = b;
        b = t;
      }
      ok = (a == 1);
    }
    if (ok) out[cnt++] = x;
  }
  return cnt;
}

// K_c: largest multiple of 256 such that every triangular partial C_s of
// Eq. (2) stays within int32 for the slice ranges (leading slice in
// [-128, 127], tails in [0, 255]), from interval products per pair.
int64_t host_chunk_len_I(int p) {
  int64_t worst = 0;
  for (int s = 0; s < p; ++s) {
    int64_t hi = 0, lo = 0;
    for (int i = 0; i <= s; ++i) {
      int64_t alo = i == 0 ? -128 : 0, ahi = i == 0 ? 127 : 255;
      int64_t blo = (s - i) == 0 ? -128 : 0, bhi = (s - i) == 0 ? 127 : 255;
      int64_t c[4] = {alo * blo, alo * bhi, ahi * blo, ahi * bhi};
      int64_t mx = c[0], mn = c[0];
      for (int q = 1; q < 4; ++q) {
        mx = c[q] > mx ? c[q] : mx;
        mn = c[q] < mn ? c[q] : mn;
      }
      hi += mx;
      lo += mn;
    }
    worst = hi > worst ? hi : worst;
    worst = -lo > worst ? -lo : worst;
  }
  int64_t lim = 2147483647LL / worst;
  return lim - lim % 256;
}

// K_c for the E4M3 engine: every |d_i d_j| <= 16 * 16, so C_s grows by at
// most (s+1) * 256 per unit of K; largest multiple of 256 keeping every FP32
// partial sum within 2^24 (where FP32 holds all integers exactly).
int64_t host_chunk_len_F8(int p) {
  int64_t worst = 0;
  for (int s = 0; s < p; ++s) worst = std::max<int64_t>(worst, static_cast<int64_t>(s + 1) * 16 * 16);
  int64_t lim = (int64_t{1} << 24) / worst;
  return lim - lim % 256;
}

namespace {
// little-endian 32-bit limb integers
using Limbs = std::vector<uint32_t>;
void limbs_mul_small(Limbs& a, uint32_t v) {
  uint64_t c = 0;
  for (auto& w : a) {
    c += static_cast<uint64_t>(w) * v;
    w = static_cast<uint32_t>(c);
    c >>= 32;
  }
  if (c) a.push_back(static_cast<uint32_t>(c));
}
uint32_t limbs_mod_small(const Limbs& a, uint32_t m) {
  uint64_t r = 0;
  for (size_t i = a.size(); i-- > 0;) r = ((r << 32) | a[i]) % m;
  return static_cast<uint32_t>(r);
}
int limbs_bitlen(const Limbs& a) {
  for (size_t i = a.size(); i-- > 0;)
    if (a[i]) {
      int b = 32;
      while (!((a[i] >> (b - 1)) & 1u)) --b;
      return static_cast<int>(32 * i) + b;
    }
  return 0;
}
Limbs limbs_P(int nm) {
  int32_t mods[kMaxModuli + 4];
  host_moduli(nm, mods);
  Limbs P{1u};
  for (int l = 0; l < nm; ++l) limbs_mul_small(P, static_cast<uint32_t>(mods[l]));
  return P;
}
// modular inverse by the extended Euclidean algorithm
int64_t inv_mod(int64_t a, int64_t m) {
  int64_t g = m, x = 0, x1 = 1, a1 = a % m;
  while (a1) {
    int64_t q = g / a1;
    int64_t t = g - q * a1;
    g = a1;
    a1 = t;
    t = x - q * x1;
    x = x1;
    x1 = t;
  }
  return ((x % m) + m) % m;
}
}  // namespace

// b = floor((floor(log2 P) - 1 - ceil(log2 k)) / 2); complex uses -2.
int host_scale_bits_II(int nm, int64_t k, int is_complex) {
  int lp = limbs_bitlen(limbs_P(nm)) - 1;
  int c = 0;
  while ((int64_t{1} << c) < k) ++c;
  int num = lp - (is_complex ? 2 : 1) - c;
  return num >= 0 ? num / 2 : -((-num + 1) / 2);
}

// Norm-based scaling: one exponent h for both operands (the product stays
// symmetric in A and B, whichever one is stored transposed), 2h + 1 <=
// floor(log2 P).
void host_norm_halves_II(int nm, int* hA, int* hB) {
  const int L = limbs_bitlen(limbs_P(nm)) - 2;  // floor(log2 P) - 1
  *hA = L >= 0 ? L / 2 : -((-L + 1) / 2);
  *hB = *hA;
}

void host_mod_tables(int nm, ModTables* t) {
  std::memset(t, 0, sizeof(*t));
  int32_t mods[kMaxModuli];
  host_moduli(nm, mods);
  for (int l = 0; l < nm; ++l) {
    const int32_t m = mods[l], hi = (m - 1) / 2;
    t->mods[l] = static_cast<uint32_t>(m);
    t->off[l] = m - 1 - hi;
    t->inv[l] = 1.0f / static_cast<float>(m);
    t->offinv[l] = static_cast<float>(t->off[l]) / static_cast<float>(m);
    t->offhinv[l] = static_cast<float>(t->off[l] + 0.5) / static_cast<float>(m);
    int64_t v = 1 % m;  // 2^(16 j) mod m
    for (int j = 0; j < kResDigits; ++j) {
      t->pow16[l][j] = static_cast<int32_t>(v > hi ? v - m : v);
      v = (v << 16) % m;
    }
    t->mf[l] = static_cast<float>(m);
    t->offf[l] = static_cast<float>(t->off[l]);
    v = 1 % m;  // 2^(14 j) mod m
    for (int j = 0; j < kResDigitsF; ++j) {
      t->pow14f[l][j] = static_cast<float>(v > hi ? v - m : v);
      v = (v << 14) % m;
    }
  }
}

void host_crt_tables(int nm, CrtTables* t) {
  std::memset(t, 0, sizeof(*t));
  int32_t mods[kMaxModuli];
  host_moduli(nm, mods);
  t->nm = nm;
  Limbs P = limbs_P(nm);
  for (int i = 0; i < kCrtLimbs && i < static_cast<int>(P.size()); ++i) t->P[i] = P[i];
  // floor(P/2)
  for (int i = 0; i < kCrtLimbs; ++i)
    t->Phalf[i] = (t->P[i] >> 1) | (i + 1 < kCrtLimbs ? (t->P[i + 1] << 31) : 0u);
  double pd = 0.0;
  for (int i = kCrtLimbs - 1; i >= 0; --i) pd = pd * 4294967296.0 + t->P[i];
  t->invP = 1.0 / pd;
  for (int l = 0; l < nm; ++l) {
    Limbs Pl{1u};
    for (int j = 0; j < nm; ++j)
      if (j != l) limbs_mul_small(Pl, static_cast<uint32_t>(mods[j]));
    uint32_t pm = limbs_mod_small(Pl, static_cast<uint32_t>(mods[l]));
    int64_t q = inv_mod(pm, mods[l]);
    limbs_mul_small(Pl, static_cast<uint32_t>(q));
    for (int i = 0; i < kCrtLimbs && i < static_cast<int>(Pl.size()); ++i) t->w[l][i] = Pl[i];
    double wd = 0.0;
    for (int i = kCrtLimbs - 1; i >= 0; --i) wd = wd * 4294967296.0 + t->w[l][i];
    t->wP[l] = static_cast<float>(wd / pd);
  }
}

// ================================================================ tensor maps
namespace {
using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                              CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                              CUtensorMapFloatOOBfill);
EncodeFn get_encode() {
  static EncodeFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeFn>(p);
  });
  return fn;
}
}  // namespace

bool make_tmap_i8(CUtensorMap* map, const void* base, uint64_t cols, uint64_t rows, uint32_t box_rows,
                  uint32_t box_bytes) {
  EncodeFn enc = get_encode();
  if (!enc) return false;
  if (box_bytes != 32 && box_bytes != 128) return false;
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {cols};
  cuuint32_t box[2] = {box_bytes, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(base), dims, strides, box,
                   estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   box_bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_32B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// ================================================================ misc kernels
template <typename T>
__global__ void scale_c_kernel(T* C, int64_t ldc, int64_t m, int64_t n, double beta) {
  int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= m * n) return;
  int64_t i = idx / n, j = idx % n;
  T* p = C + i * ldc + j;
  *p = beta == 0.0 ? T(0) : static_cast<T>(__dmul_rn(beta, static_cast<double>(*p)));
}
// k == 0: C = beta * C for complex beta (C not read when beta == 0); float
// C (CGEMM) is widened, updated in binary64 and rounded once per part.
template <typename T>
__global__ void scale_z_kernel(T* C, int64_t ldc, int64_t m, int64_t n, double br, double bi) {
  int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= m * n) return;
  int64_t i = idx / n, j = idx % n;
  T* p = C + 2 * (i * ldc + j);
  if (br == 0.0 && bi == 0.0) {
    p[0] = T(0);
    p[1] = T(0);
    return;
  }
  double cr = static_cast<double>(p[0]), ci = static_cast<double>(p[1]);
  p[0] = static_cast<T>(__fma_rn(br, cr, -__dmul_rn(bi, ci)));
  p[1] = static_cast<T>(__fma_rn(br, ci, __dmul_rn(bi, cr)));
}

// One warp waits on an mbarrier that nothing arrives on; the bounded wait
// gives up after `limit` cycles and records the timeout.
__global__ void selftest_wait_kernel(int* status, long long limit) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncwarp();
  if (threadIdx.x == 0 && !mbar_wait_bounded(&bar, 0, limit)) set_status(status, ST_TIMEOUT);
}

}  // namespace emu

using namespace emu;

// ================================================================ handle
// What was behind this thread's last EMU_ERR_CUDA (emu_last_cuda_error).
static thread_local const char* g_last_cuda_error = "no error";
static emu_status_t cuda_err(cudaError_t e) {
  if (e == cudaSuccess) return EMU_OK;
  g_last_cuda_error = cudaGetErrorString(e);
  return EMU_ERR_CUDA;
}
static emu_status_t tmap_err() {
  g_last_cuda_error = "tensor map encoding failed";
  return EMU_ERR_CUDA;
}

namespace emu {
// EMU_FAULT=alloc / EMU_FAULT=launch: host-side fault injection (read once).
static int fault_mode() {
  static int v = -1;
  if (v < 0) {
    const char* e = std::getenv("EMU_FAULT");
    v = !e ? 0 : std::strcmp(e, "alloc") == 0 ? 1 : std::strcmp(e, "launch") == 0 ? 2 : 0;
  }
  return v;
}
// alloc: every library-owned workspace allocation fails.
static bool fault_alloc() { return fault_mode() == 1; }
// launch: the fused GEMM launch of every product fails as a launch would
// (cudaErrorLaunchFailure, after the scan and split were enqueued); nothing
// runs on the device that could fault.
static cudaError_t fault_launch() { return fault_mode() == 2 ? cudaErrorLaunchFailure : cudaSuccess; }

emu_status_t handle_workspace(emu_handle_s* h, size_t bytes, cudaStream_t st, uint8_t** out) {
  if (bytes == 0) bytes = 256;
  if (!h->ws_user && bytes > h->ws_bytes && fault_alloc()) return EMU_ERR_ALLOC;
  if (h->ws_user) {
    if (bytes > h->ws_bytes) return EMU_ERR_ALLOC;
    *out = static_cast<uint8_t*>(h->ws);
    return EMU_OK;
  }
  if (bytes > h->ws_bytes) {
    // no growth inside a stream capture: the memory would belong to the
    // graph, and the handle would keep using it after the capture
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
      cudaGetLastError();
      return EMU_ERR_ALLOC;
    }
    if (h->ws) cudaFreeAsync(h->ws, st);
    h->ws = nullptr;
    h->ws_bytes = 0;
    size_t want = bytes + bytes / 8;
    if (cudaMallocAsync(&h->ws, want, st) != cudaSuccess) {
      h->ws = nullptr;
      cudaGetLastError();
      return EMU_ERR_ALLOC;
    }
    h->ws_bytes = want;
  }
  *out = static_cast<uint8_t*>(h->ws);
  return EMU_OK;
}
}  // namespace emu

extern "C" {

emu_status_t emu_create(emu_handle_t* out, int device) {
  if (!out) return EMU_ERR_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return EMU_ERR_CUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) return EMU_ERR_CUDA;
  emu_handle_s* h = new (std::nothrow) emu_handle_s();
  if (!h) return EMU_ERR_ALLOC;
  h->device = device;
  cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (cudaMalloc(&h->status, sizeof(int)) != cudaSuccess) {
    delete h;
    return EMU_ERR_ALLOC;
  }
  cudaMemset(h->status, 0, sizeof(int));
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaFree(h->status);
    delete h;
    return EMU_ERR_CUDA;
  }
  *out = h;
  return EMU_OK;
}

emu_status_t emu_destroy(emu_handle_t h) {
  if (!h) return EMU_OK;
  cudaSetDevice(h->device);
  cudaDeviceSynchronize();
  handle_release_extras(h);
  if (h->ws && !h->ws_user) cudaFree(h->ws);
  if (h->status) cudaFree(h->status);
  delete h;
  return EMU_OK;
}

emu_status_t emu_get_status(emu_handle_t h, emu_stream_t stream) {
  if (!h) return EMU_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaStreamSynchronize(st) != cudaSuccess) return EMU_ERR_CUDA;
  int v = 0;
  if (cudaMemcpy(&v, h->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return EMU_ERR_CUDA;
  cudaMemset(h->status, 0, sizeof(int));
  cudaDeviceSynchronize();
  if (v & ST_TIMEOUT) return EMU_ERR_TIMEOUT;
  if (v & ST_NONFINITE) return EMU_ERR_NONFINITE;
  return EMU_OK;
}

emu_status_t emu_selftest_wait(emu_handle_t h, int64_t limit_cycles, emu_stream_t stream) {
  if (!h) return EMU_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  long long lim = limit_cycles < 1000 ? 1000 : (limit_cycles > 2000000000LL ? 2000000000LL : limit_cycles);
  selftest_wait_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(h->status, lim);
  return cuda_err(cudaGetLastError());
}

const char* emu_last_cuda_error(void) { return g_last_cuda_error; }

const char* emu_status_string(emu_status_t s) {
  switch (s) {
    case EMU_OK: return "EMU_OK";
    case EMU_ERR_INVALID_ARG: return "EMU_ERR_INVALID_ARG";
    case EMU_ERR_UNSUPPORTED: return "EMU_ERR_UNSUPPORTED";
    case EMU_ERR_NONFINITE: return "EMU_ERR_NONFINITE";
    case EMU_ERR_CUDA: return "EMU_ERR_CUDA";
    case EMU_ERR_ALLOC: return "EMU_ERR_ALLOC";
    case EMU_ERR_TIMEOUT: return "EMU_ERR_TIMEOUT";
    case EMU_ERR_TOL_NOT_MET: return "EMU_ERR_TOL_NOT_MET";
  }
  return "EMU_ERR_UNKNOWN";
}

int64_t emu_split_rows(int64_t rows) { return split_rows(rows); }
int64_t emu_split_cols_I(int64_t k, int p) { return split_cols_I(k, p); }
int64_t emu_split_cols_II(int64_t k) { return split_cols_II(k); }
int64_t emu_chunk_len_I(int p) { return p >= 1 ? host_chunk_len_I(p) : 0; }
int64_t emu_chunk_len_F8(int p) { return p >= 1 ? host_chunk_len_F8(p) : 0; }
int emu_moduli(int nm, int32_t* mods) { return mods ? host_moduli(nm, mods) : 0; }
int emu_scale_bits_II(int nm, int64_t k, int is_complex) { return host_scale_bits_II(nm, k, is_complex); }

emu_status_t emu_set_workspace(emu_handle_t h, void* ws, size_t bytes) {
  if (!h) return EMU_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  if (h->ws && !h->ws_user) {
    cudaDeviceSynchronize();
    cudaFree(h->ws);
  }
  h->ws = ws;
  h->ws_bytes = ws ? bytes : 0;
  h->ws_user = ws != nullptr;
  if (ws && (reinterpret_cast<uintptr_t>(ws) & 255u)) return EMU_ERR_INVALID_ARG;
  return EMU_OK;
}

}  // extern "C"

// ================================================================ planning
namespace emu {

static inline size_t al256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

// EMU_F8_ENGINE=mma selects the warp-level FP8 kernel for E4M3 slices (for
// comparison); the default is the tcgen05 kernel.
static bool f8_engine_mma() {
  static int v = -1;
  if (v < 0) {
    const char* e = std::getenv("EMU_F8_ENGINE");
    v = (e && std::strcmp(e, "mma") == 0) ? 1 : 0;
  }
  return v == 1;
}

// EMU_II_ENGINE=mma selects the INT8 mma.sync kernel for Scheme II (for
// comparison; identical results); the default is the bf16 tcgen05 kernel.
bool ii_engine_tc() {
  static int v = -1;
  if (v < 0) {
    const char* e = std::getenv("EMU_II_ENGINE");
    v = (e && std::strcmp(e, "mma") == 0) ? 0 : 1;
  }
  return v == 1;
}

Plan plan_I(int64_t m, int64_t n, int64_t k, int p) {
  Plan pl{};
  pl.rows_a = split_rows(m);
  pl.rows_b = split_rows(n);
  pl.cols = split_cols_I(k, p);
  size_t off = 0;
  pl.off_maxA = off; off += al256(8 * static_cast<size_t>(m > 0 ? m : 1));
  pl.off_maxB = off; off += al256(8 * static_cast<size_t>(n > 0 ? n : 1));
  pl.off_EA = off; off += al256(4 * static_cast<size_t>(m > 0 ? m : 1));
  pl.off_FB = off; off += al256(4 * static_cast<size_t>(n > 0 ? n : 1));
  pl.off_hatA = off; off += al256(static_cast<size_t>(pl.rows_a) * pl.cols);
  pl.off_hatB = off; off += al256(static_cast<size_t>(pl.rows_b) * pl.cols);
  pl.bytes = off;
  return pl;
}

// es: bytes per residue (1: INT8 planes, 2: bf16 planes of the tcgen05 kernel)
Plan plan_II(int64_t m, int64_t n, int64_t k, int nm, int nsets, int es) {
  Plan pl{};
  pl.rows_a = split_rows(m);
  pl.rows_b = split_rows(n);
  pl.cols = split_cols_II(k);
  size_t off = 0;
  pl.off_maxA = off; off += al256(8 * static_cast<size_t>(m > 0 ? m : 1));
  pl.off_maxB = off; off += al256(8 * static_cast<size_t>(n > 0 ? n : 1));
  pl.off_EA = off; off += al256(4 * static_cast<size_t>(m > 0 ? m : 1));
  pl.off_FB = off; off += al256(4 * static_cast<size_t>(n > 0 ? n : 1));
  pl.off_hatA = off; off += al256(static_cast<size_t>(es) * nsets * nm * pl.rows_a * pl.cols);
  pl.off_hatB = off; off += al256(static_cast<size_t>(es) * nsets * nm * pl.rows_b * pl.cols);
  // norm-based scaling: 128-bit sums of squares and the exponents
  pl.off_accA = off; off += al256(16 * static_cast<size_t>(m > 0 ? m : 1));
  pl.off_accB = off; off += al256(16 * static_cast<size_t>(n > 0 ? n : 1));
  pl.off_nEA = off; off += al256(4 * static_cast<size_t>(m > 0 ? m : 1));
  pl.off_nEB = off; off += al256(4 * static_cast<size_t>(n > 0 ? n : 1));
  // tcgen05 kernel: the residue planes (one byte per output and modulus; row
  // tiles rounded to whole CTA-pair tiles)
  pl.off_scratch = off; off += es == 2 ? al256(gemm_II_tc_residue_bytes(m, n, nm, nsets == 3, 2)) : 0;
  pl.bytes = off;
  return pl;
}

// Row-major view of the product: C (M x N) = Aop (M x K) * Bop (K x N) where
// Aop's rows are reduction vectors read with (ldA, a_kcontig) and Bop's
// columns with (ldB, b_kcontig).  Column-major calls are mapped onto the
// transposed row-major product C^T = B^T A^T.
void normalize(emu_layout_t layout, int64_t m, int64_t n, const void* A, int64_t lda, const void* B,
               int64_t ldb, View* v) {
  if (layout == EMU_ROW_MAJOR) {
    v->M = m;
    v->N = n;
    v->A = A;
    v->ldA = lda;
    v->a_kcontig = true;
    v->B = B;
    v->ldB = ldb;
    v->b_kcontig = false;
  } else {
    v->M = n;
    v->N = m;
    v->A = B;
    v->ldA = ldb;
    v->a_kcontig = true;
    v->B = A;
    v->ldB = lda;
    v->b_kcontig = false;
  }
}

bool check_lds(emu_layout_t layout, int64_t m, int64_t n, int64_t k, int64_t lda, int64_t ldb,
               int64_t ldc) {
  if (layout == EMU_ROW_MAJOR)
    return lda >= (k > 1 ? k : 1) && ldb >= (n > 1 ? n : 1) && ldc >= (n > 1 ? n : 1);
  return lda >= (m > 1 ? m : 1) && ldb >= (k > 1 ? k : 1) && ldc >= (m > 1 ? m : 1);
}

template <typename T>
emu_status_t run_scheme_I(emu_handle_s* h, const View& v, int64_t k, int p, double alpha, double beta,
                          void* C, int64_t ldc, int out_mode, int32_t* partials, cudaStream_t st,
                          uint8_t* ws_override, bool f8) {
  Plan pl = plan_I(v.M, v.N, k, p);
  uint8_t* ws = ws_override;
  if (!ws) {
    emu_status_t s = handle_workspace(h, pl.bytes, st, &ws);
    if (s != EMU_OK) return s;
  }
  auto* maxA = reinterpret_cast<unsigned long long*>(ws + pl.off_maxA);
  auto* maxB = reinterpret_cast<unsigned long long*>(ws + pl.off_maxB);
  auto* EA = reinterpret_cast<int32_t*>(ws + pl.off_EA);
  auto* FB = reinterpret_cast<int32_t*>(ws + pl.off_FB);
  auto* hatA = reinterpret_cast<int8_t*>(ws + pl.off_hatA);
  auto* hatB = reinterpret_cast<int8_t*>(ws + pl.off_hatB);
  const T* A = static_cast<const T*>(v.A);
  const T* B = static_cast<const T*>(v.B);
  trace_begin(h, PH_SCAN, st);
  launch_scan<T>(A, v.ldA, v.a_kcontig, v.M, k, 1, maxA, h->status, st);
  launch_scan<T>(B, v.ldB, v.b_kcontig, v.N, k, 1, maxB, h->status, st);
  trace_end(h, PH_SCAN, st, 2);
  trace_begin(h, PH_SPLIT, st);
  launch_split_I<T>(A, v.ldA, v.a_kcontig, v.M, k, p, maxA, hatA, EA, st, f8);
  launch_split_I<T>(B, v.ldB, v.b_kcontig, v.N, k, p, maxB, hatB, FB, st, f8);
  trace_end(h, PH_SPLIT, st, 2);
  return scheme_I_gemm(h, hatA, pl.rows_a, hatB, pl.rows_b, pl.cols, v.M, v.N, k, p, EA, FB, alpha, beta, C, ldc,
                       out_mode, partials, st, f8);
}

// The fused Scheme I GEMM on split operands: hatA (rows_a padded rows) and
// hatB (rows_b) in the interleaved slice layout, `cols` bytes per row; C
// (M x N, leading dimension ldc) from the exact slice sums scaled by EA (M)
// and FB (N).
emu_status_t scheme_I_gemm(emu_handle_s* h, const int8_t* hatA, int64_t rows_a, const int8_t* hatB, int64_t rows_b,
                           int64_t cols, int64_t M, int64_t N, int64_t k, int p, const int32_t* EA,
                           const int32_t* FB, double alpha, double beta, void* C, int64_t ldc, int out_mode,
                           int32_t* partials, cudaStream_t st, bool f8) {
  // E4M3 slices run on the tcgen05 kernel (A boxes of 128 B x 128 rows);
  // the INT8 engine uses the mma.sync kernel (32 B x 64 rows).
  const bool tc = f8 && !f8_engine_mma();
  CUtensorMap ta, tb;
  if (!make_tmap_i8(&ta, hatA, static_cast<uint64_t>(cols), static_cast<uint64_t>(rows_a),
                    tc ? 128u : 64u, tc ? 128 : 32) ||
      !make_tmap_i8(&tb, hatB, static_cast<uint64_t>(cols), static_cast<uint64_t>(rows_b), 32))
    return tmap_err();
  GemmIArgs a{};
  a.descA = &ta;
  a.descB = &tb;
  a.M = static_cast<int>(M);
  a.N = static_cast<int>(N);
  a.nk32 = static_cast<int>((k + 31) / 32);
  a.kc32 = static_cast<int>((f8 ? host_chunk_len_F8(p) : host_chunk_len_I(p)) / 32);
  a.EA = EA;
  a.FB = FB;
  a.alpha = alpha;
  a.beta = beta;
  a.C = C;
  a.ldc = ldc;
  a.partials = partials;
  a.status = h->status;
  a.num_sms = h->num_sms;
  trace_begin(h, PH_GEMM, st);
  cudaError_t e = fault_launch();
  if (e == cudaSuccess) e = tc ? launch_gemm_f8tc(p, out_mode, a, st) : launch_gemm_I(p, out_mode, a, st, f8);
  trace_end(h, PH_GEMM, st, 1);
  return cuda_err(e);
}
template emu_status_t run_scheme_I<double>(emu_handle_s*, const View&, int64_t, int, double, double,
                                           void*, int64_t, int, int32_t*, cudaStream_t, uint8_t*, bool);
template emu_status_t run_scheme_I<float>(emu_handle_s*, const View&, int64_t, int, double, double,
                                          void*, int64_t, int, int32_t*, cudaStream_t, uint8_t*, bool);

template <typename T>
// Phases (declared in emu_handle.h): B's split once, then A in row chunks
// (per-row scaling makes the chunks independent).
emu_status_t run_scheme_II(emu_handle_s* h, const View& v, int64_t k, int nm, int cw, double ar,
                           double ai, double br, double bi, void* C, int64_t ldc, int out_mode,
                           uint8_t* residues, cudaStream_t st, bool norm, int phase, int64_t plan_rows) {
  const int nsets = cw == 2 ? 3 : 1;
  // the tcgen05 kernel takes bf16 residue planes; the INT8 kernel sums a
  // modulus's products over the whole K in INT32 (|sum| <= k 2^14)
  const bool tc = out_mode != II_RESIDUES && ii_engine_tc();
  if (!tc && k > EMU_K_MAX_II) return EMU_ERR_UNSUPPORTED;
  Plan pl = plan_II(plan_rows > 0 ? plan_rows : v.M, v.N, k, nm, nsets, tc ? 2 : 1);
  pl.rows_a = split_rows(v.M);  // A's planes are laid out for this call's rows
  uint8_t* ws = nullptr;
  emu_status_t s = handle_workspace(h, pl.bytes, st, &ws);
  if (s != EMU_OK) return s;
  auto* maxA = reinterpret_cast<unsigned long long*>(ws + pl.off_maxA);
  auto* maxB = reinterpret_cast<unsigned long long*>(ws + pl.off_maxB);
  auto* EA = reinterpret_cast<int32_t*>(ws + pl.off_EA);
  auto* FB = reinterpret_cast<int32_t*>(ws + pl.off_FB);
  auto* resA = reinterpret_cast<int8_t*>(ws + pl.off_hatA);
  auto* resB = reinterpret_cast<int8_t*>(ws + pl.off_hatB);
  const T* A = static_cast<const T*>(v.A);
  const T* B = static_cast<const T*>(v.B);
  // worst-case scaling (one b for both operands, exponents of the row
  // maxima) or norm-based scaling (hA, hB, exponents of the 2-norms)
  int bA = host_scale_bits_II(nm, k, cw == 2), bB = bA;
  if (norm) host_norm_halves_II(nm, &bA, &bB);
  auto* nEA = reinterpret_cast<int32_t*>(ws + pl.off_nEA);
  auto* nEB = reinterpret_cast<int32_t*>(ws + pl.off_nEB);
  ModTables mt;
  host_mod_tables(nm, &mt);
  CrtTables ct;
  host_crt_tables(nm, &ct);
  const bool do_a = phase != 1, do_b = phase != 2;
  trace_begin(h, PH_SCAN, st);
  if (do_a) launch_scan<T>(A, v.ldA, v.a_kcontig, v.M, k, cw, maxA, h->status, st);
  if (do_b) launch_scan<T>(B, v.ldB, v.b_kcontig, v.N, k, cw, maxB, h->status, st);
  if (norm && do_a)
    launch_norm<T>(A, v.ldA, v.a_kcontig, v.M, k, cw, maxA, reinterpret_cast<unsigned long long*>(ws + pl.off_accA),
                   nEA, st);
  if (norm && do_b)
    launch_norm<T>(B, v.ldB, v.b_kcontig, v.N, k, cw, maxB, reinterpret_cast<unsigned long long*>(ws + pl.off_accB),
                   nEB, st);
  trace_end(h, PH_SCAN, st, (do_a + do_b) * (norm ? 3 : 1));
  trace_begin(h, PH_SPLIT, st);
  if (do_a)
    launch_split_II<T>(A, v.ldA, v.a_kcontig, v.M, k, nm, bA, cw, mt, maxA, resA, EA, st, norm ? nEA : nullptr, tc);
  if (do_b)
    launch_split_II<T>(B, v.ldB, v.b_kcontig, v.N, k, nm, bB, cw, mt, maxB, resB, FB, st, norm ? nEB : nullptr, tc);
  trace_end(h, PH_SPLIT, st, do_a + do_b);
  if (phase == 1) return cuda_err(cudaGetLastError());
  CUtensorMap ta, tb;
  // tcgen05: the bf16 planes as bytes, 128-byte (64-element) boxes of 128
  // rows (A) and 256 / cluster rows (B: a CTA pair loads half of each
  // 256-column tile per CTA); INT8: 32-byte boxes of 64 / 32 rows
  const uint64_t row_bytes = static_cast<uint64_t>(pl.cols) * (tc ? 2 : 1);
  const int cluster = tc ? gemm_II_tc_cluster() : 1;
  if (!make_tmap_i8(&ta, resA, row_bytes, static_cast<uint64_t>(pl.rows_a) * nm * nsets,
                    tc ? static_cast<uint32_t>(gemm_II_tc_tile_m()) : 64, tc ? 128 : 32) ||
      !make_tmap_i8(&tb, resB, row_bytes, static_cast<uint64_t>(pl.rows_b) * nm * nsets,
                    tc ? static_cast<uint32_t>(gemm_II_tc_tile_n() / cluster) : 32, tc ? 128 : 32))
    return tmap_err();
  GemmIIArgs a{};
  a.descA = &ta;
  a.descB = &tb;
  a.M = static_cast<int>(v.M);
  a.N = static_cast<int>(v.N);
  a.nk32 = static_cast<int>(pl.cols / 32);
  a.rowsA_pad = static_cast<int>(pl.rows_a);
  a.rowsB_pad = static_cast<int>(pl.rows_b);
  a.nm = nm;
  a.escale = -(bA + bB);
  a.EA = EA;
  a.FB = FB;
  a.alpha_re = ar;
  a.alpha_im = ai;
  a.beta_re = br;
  a.beta_im = bi;
  a.C = C;
  a.ldc = ldc;
  a.residues = residues;
  a.status = h->status;
  a.num_sms = h->num_sms;
  a.cluster = cluster;
  a.scratch = ws + pl.off_scratch;
  if (!tc) {
    trace_begin(h, PH_GEMM, st);
    cudaError_t e = fault_launch();
    if (e == cudaSuccess) e = launch_gemm_II(out_mode, a, mt, ct, st);
    trace_end(h, PH_GEMM, st, 1);
    return cuda_err(e);
  }
  // the residue GEMM is the traced GEMM phase, the CRT kernel "other"
  trace_begin(h, PH_GEMM, st);
  cudaError_t e = fault_launch();
  if (e == cudaSuccess) e = launch_gemm_II_tc(out_mode, a, mt, ct, st, 1);
  trace_end(h, PH_GEMM, st, 1);
  if (e != cudaSuccess) return cuda_err(e);
  trace_begin(h, PH_OTHER, st);
  e = launch_gemm_II_tc(out_mode, a, mt, ct, st, 2);
  trace_end(h, PH_OTHER, st, 1);
  return cuda_err(e);
}

template emu_status_t run_scheme_II<double>(emu_handle_s*, const View&, int64_t, int, int, double, double, double,
                                            double, void*, int64_t, int, uint8_t*, cudaStream_t, bool, int, int64_t);
template emu_status_t run_scheme_II<float>(emu_handle_s*, const View&, int64_t, int, int, double, double, double,
                                           double, void*, int64_t, int, uint8_t*, cudaStream_t, bool, int, int64_t);

template <typename T>
void launch_scale_c(T* C, int64_t ldc, int64_t M, int64_t N, double beta, cudaStream_t st) {
  int64_t tot = M * N;
  if (tot <= 0) return;
  scale_c_kernel<T><<<static_cast<unsigned>((tot + 255) / 256), 256, 0, st>>>(C, ldc, M, N, beta);
}
template void launch_scale_c<double>(double*, int64_t, int64_t, int64_t, double, cudaStream_t);

}  // namespace emu

// ================================================================ entry points
extern "C" {

emu_status_t emu_workspace_size(emu_scheme_t scheme, int64_t m, int64_t n, int64_t k, int p_or_nm,
                                int is_complex, size_t* bytes) {
  if (!bytes || m < 0 || n < 0 || k < 0) return EMU_ERR_INVALID_ARG;
  if (scheme == EMU_SCHEME_I || scheme == EMU_SCHEME_I_F8) {
    if (p_or_nm < EMU_P_MIN || p_or_nm > EMU_P_MAX) return EMU_ERR_UNSUPPORTED;
    *bytes = is_complex ? workspace_complex_I(m, n, k, p_or_nm) : plan_I(m, n, k, p_or_nm).bytes;
    return EMU_OK;
  }
  if (scheme == EMU_SCHEME_II || scheme == EMU_SCHEME_II_NORM) {
    if (p_or_nm < EMU_NM_MIN || p_or_nm > EMU_NM_MAX) return EMU_ERR_UNSUPPORTED;
    *bytes = plan_II(m, n, k, p_or_nm, is_complex ? 3 : 1, ii_engine_tc() ? 2 : 1).bytes;
    return EMU_OK;
  }
  return EMU_ERR_INVALID_ARG;
}

}  // extern "C"

emu_status_t emu::gemm_common(emu_handle_t h, emu_layout_t layout, int64_t m, int64_t n, int64_t k,
                                const void* A, int64_t lda, const void* B, int64_t ldb, const void* C,
                                int64_t ldc, emu_scheme_t scheme, int p_or_nm) {
  if (!h) return EMU_ERR_INVALID_ARG;
  if (layout != EMU_ROW_MAJOR && layout != EMU_COL_MAJOR) return EMU_ERR_INVALID_ARG;
  if (m < 0 || n < 0 || k < 0) return EMU_ERR_INVALID_ARG;
  if (m > INT32_MAX / 2 || n > INT32_MAX / 2 || k > (int64_t{1} << 30)) return EMU_ERR_UNSUPPORTED;
  if (!check_lds(layout, m, n, k, lda, ldb, ldc)) return EMU_ERR_INVALID_ARG;
  if (m > 0 && n > 0 && !C) return EMU_ERR_INVALID_ARG;
  if (m > 0 && n > 0 && k > 0 && (!A || !B)) return EMU_ERR_INVALID_ARG;
  if (scheme == EMU_SCHEME_I || scheme == EMU_SCHEME_I_F8) {
    if (p_or_nm < EMU_P_MIN || p_or_nm > EMU_P_MAX) return EMU_ERR_UNSUPPORTED;
  } else if (scheme == EMU_SCHEME_II || scheme == EMU_SCHEME_II_NORM) {
    if (p_or_nm < EMU_NM_MIN || p_or_nm > EMU_NM_MAX) return EMU_ERR_UNSUPPORTED;
    if (k > EMU_K_MAX_II && !ii_engine_tc()) return EMU_ERR_UNSUPPORTED;
  } else {
    return EMU_ERR_INVALID_ARG;
  }
  if (cudaSetDevice(h->device) != cudaSuccess) return EMU_ERR_CUDA;
  return EMU_OK;
}

template <typename T>
static emu_status_t real_gemm(emu_handle_t h, emu_layout_t layout, int64_t m, int64_t n, int64_t k,
                              double alpha, const T* A, int64_t lda, const T* B, int64_t ldb,
                              double beta, T* C, int64_t ldc, emu_scheme_t scheme, int p_or_nm,
                              emu_stream_t stream) {
  emu_status_t s = gemm_common(h, layout, m, n, k, A, lda, B, ldb, C, ldc, scheme, p_or_nm);
  if (s != EMU_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  View v;
  normalize(layout, m, n, A, lda, B, ldb, &v);
  if (v.M == 0 || v.N == 0) return EMU_OK;
  if (k == 0) {
    launch_scale_c<T>(C, ldc, v.M, v.N, beta, st);
    return cuda_err(cudaGetLastError());
  }
  const int out = sizeof(T) == 8 ? 0 : 1;
  if (scheme == EMU_SCHEME_I || scheme == EMU_SCHEME_I_F8)
    return run_scheme_I<T>(h, v, k, p_or_nm, alpha, beta, C, ldc, out == 0 ? OUT_F64 : OUT_F32, nullptr,
                           st, nullptr, scheme == EMU_SCHEME_I_F8);
  return run_scheme_II<T>(h, v, k, p_or_nm, 1, alpha, 0.0, beta, 0.0, C, ldc, out == 0 ? II_F64 : II_F32,
                          nullptr, st, scheme == EMU_SCHEME_II_NORM);
}

extern "C" {

emu_status_t emu_dgemm(emu_handle_t h, emu_layout_t layout, int64_t m, int64_t n, int64_t k, double alpha,
                       const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C,
                       int64_t ldc, emu_scheme_t scheme, int p_or_nm, emu_stream_t stream) {
  return real_gemm<double>(h, layout, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, scheme, p_or_nm, stream);
}

emu_status_t emu_sgemm(emu_handle_t h, emu_layout_t layout, int64_t m, int64_t n, int64_t k, float alpha,
                       const float* A, int64_t lda, const float* B, int64_t ldb, float beta, float* C,
                       int64_t ldc, emu_scheme_t scheme, int p_or_nm, emu_stream_t stream) {
  return real_gemm<float>(h, layout, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, scheme, p_or_nm, stream);
}

emu_status_t emu_zgemm(emu_handle_t h, emu_layout_t layout, int64_t m, int64_t n, int64_t k,
                       const double* alpha, const double* A, int64_t lda, const double* B, int64_t ldb,
                       const double* beta, double* C, int64_t ldc, emu_scheme_t scheme, int nm,
                       emu_stream_t stream) {
  if (!alpha || !beta) return EMU_ERR_INVALID_ARG;
  emu_status_t s = gemm_common(h, layout, m, n, k, A, lda, B, ldb, C, ldc, scheme, nm);
  if (s != EMU_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  View v;
  normalize(layout, m, n, A, lda, B, ldb, &v);
  if (v.M == 0 || v.N == 0) return EMU_OK;
  if (k == 0) {
    int64_t tot = v.M * v.N;
    scale_z_kernel<double>
        <<<static_cast<unsigned>((tot + 255) / 256), 256, 0, st>>>(C, ldc, v.M, v.N, beta[0], beta[1]);
    return cuda_err(cudaGetLastError());
  }
  if (scheme == EMU_SCHEME_I || scheme == EMU_SCHEME_I_F8)
    return run_complex_I<double>(h, layout, m, n, k, A, lda, B, ldb, nm, scheme == EMU_SCHEME_I_F8, alpha, beta,
                                 C, ldc, st);
  return run_scheme_II<double>(h, v, k, nm, 2, alpha[0], alpha[1], beta[0], beta[1], C, ldc, II_Z3M,
                               nullptr, st, scheme == EMU_SCHEME_II_NORM);
}

emu_status_t emu_cgemm(emu_handle_t h, emu_layout_t layout, int64_t m, int64_t n, int64_t k,
                       const float* alpha, const float* A, int64_t lda, const float* B, int64_t ldb,
                       const float* beta, float* C, int64_t ldc, emu_scheme_t scheme, int p_or_nm,
                       emu_stream_t stream) {
  if (!alpha || !beta) return EMU_ERR_INVALID_ARG;
  emu_status_t s = gemm_common(h, layout, m, n, k, A, lda, B, ldb, C, ldc, scheme, p_or_nm);
  if (s != EMU_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  View v;
  normalize(layout, m, n, A, lda, B, ldb, &v);
  if (v.M == 0 || v.N == 0) return EMU_OK;
  const double al[2] = {alpha[0], alpha[1]}, be[2] = {beta[0], beta[1]};
  if (k == 0) {
    int64_t tot = v.M * v.N;
    scale_z_kernel<float>
        <<<static_cast<unsigned>((tot + 255) / 256), 256, 0, st>>>(C, ldc, v.M, v.N, be[0], be[1]);
    return cuda_err(cudaGetLastError());
  }
  if (scheme == EMU_SCHEME_II || scheme == EMU_SCHEME_II_NORM)
    return run_scheme_II<float>(h, v, k, p_or_nm, 2, al[0], al[1], be[0], be[1], C, ldc, II_C3M, nullptr, st,
                                scheme == EMU_SCHEME_II_NORM);
  return run_complex_I<float>(h, layout, m, n, k, A, lda, B, ldb, p_or_nm, scheme == EMU_SCHEME_I_F8, al, be, C,
                              ldc, st);
}

// ---------------------------------------------------------------- steps
static emu_status_t split_slices(emu_handle_t h, emu_layout_t layout, int operand, int64_t rows, int64_t k,
                                 const double* X, int64_t ldx, int p, int8_t* hat, int32_t* E, emu_stream_t stream,
                                 bool f8);

emu_status_t emu_split_I(emu_handle_t h, emu_layout_t layout, int operand, int64_t rows, int64_t k,
                         const double* X, int64_t ldx, int p, int8_t* hat, int32_t* E, emu_stream_t stream) {
  return split_slices(h, layout, operand, rows, k, X, ldx, p, hat, E, stream, false);
}

emu_status_t emu_split_F8(emu_handle_t h, emu_layout_t layout, int operand, int64_t rows, int64_t k,
                          const double* X, int64_t ldx, int p, int8_t* hat, int32_t* E, emu_stream_t stream) {
  return split_slices(h, layout, operand, rows, k, X, ldx, p, hat, E, stream, true);
}

}  // extern "C"

static emu_status_t split_slices(emu_handle_t h, emu_layout_t layout, int operand, int64_t rows, int64_t k,
                                 const double* X, int64_t ldx, int p, int8_t* hat, int32_t* E, emu_stream_t stream,
                                 bool f8) {
  if (!h || !hat || !E || rows < 0 || k < 0 || (operand != 0 && operand != 1)) return EMU_ERR_INVALID_ARG;
  if (layout != EMU_ROW_MAJOR && layout != EMU_COL_MAJOR) return EMU_ERR_INVALID_ARG;
  if (p < EMU_P_MIN || p > EMU_P_MAX) return EMU_ERR_UNSUPPORTED;
  if (rows > 0 && k > 0 && !X) return EMU_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // operand 0: X is rows x k (A); operand 1: X is k x rows (B)
  bool kcontig = (operand == 0) == (layout == EMU_ROW_MAJOR);
  if (ldx < 1) return EMU_ERR_INVALID_ARG;
  uint8_t* ws = nullptr;
  emu_status_t s = handle_workspace(h, 8 * static_cast<size_t>(rows > 0 ? rows : 1), st, &ws);
  if (s != EMU_OK) return s;
  auto* mx = reinterpret_cast<unsigned long long*>(ws);
  launch_scan<double>(X, ldx, kcontig, rows, k, 1, mx, h->status, st);
  launch_split_I<double>(X, ldx, kcontig, rows, k, p, mx, hat, E, st, f8);
  return cuda_err(cudaGetLastError());
}

extern "C" {

emu_status_t emu_split_II(emu_handle_t h, emu_layout_t layout, int operand, int64_t rows, int64_t k,
                          int64_t k_total, const double* X, int64_t ldx, int nm, int8_t* res, int32_t* E,
                          emu_stream_t stream) {
  if (!h || !res || !E || rows < 0 || k < 0 || (operand != 0 && operand != 1)) return EMU_ERR_INVALID_ARG;
  if (layout != EMU_ROW_MAJOR && layout != EMU_COL_MAJOR) return EMU_ERR_INVALID_ARG;
  if (nm < EMU_NM_MIN || nm > EMU_NM_MAX) return EMU_ERR_UNSUPPORTED;
  if ((rows > 0 && k > 0 && !X) || ldx < 1) return EMU_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  bool kcontig = (operand == 0) == (layout == EMU_ROW_MAJOR);
  uint8_t* ws = nullptr;
  emu_status_t s = handle_workspace(h, 8 * static_cast<size_t>(rows > 0 ? rows : 1), st, &ws);
  if (s != EMU_OK) return s;
  auto* mx = reinterpret_cast<unsigned long long*>(ws);
  ModTables mt;
  host_mod_tables(nm, &mt);
  int b = host_scale_bits_II(nm, k_total, 0);
  launch_scan<double>(X, ldx, kcontig, rows, k, 1, mx, h->status, st);
  launch_split_II<double>(X, ldx, kcontig, rows, k, nm, b, 1, mt, mx, res, E, st);
  return cuda_err(cudaGetLastError());
}

emu_status_t emu_partials_I(emu_handle_t h, emu_layout_t layout, int64_t m, int64_t n, int64_t k,
                            const double* A, int64_t lda, const double* B, int64_t ldb, int p, int32_t* Cs,
                            emu_stream_t stream) {
  emu_status_t s = gemm_common(h, layout, m, n, k, A, lda, B, ldb, Cs, layout == EMU_ROW_MAJOR ? n : m,
                               EMU_SCHEME_I, p);
  if (s != EMU_OK) return s;
  if (k > host_chunk_len_I(p)) return EMU_ERR_UNSUPPORTED;
  if (layout != EMU_ROW_MAJOR) return EMU_ERR_UNSUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  View v;
  normalize(layout, m, n, A, lda, B, ldb, &v);
  if (v.M == 0 || v.N == 0) return EMU_OK;
  if (k == 0) return cuda_err(cudaMemsetAsync(Cs, 0, sizeof(int32_t) * p * v.M * v.N, st));
  return run_scheme_I<double>(h, v, k, p, 1.0, 0.0, nullptr, 0, OUT_PARTIALS, Cs, st, nullptr);
}

emu_status_t emu_partials_F8(emu_handle_t h, emu_layout_t layout, int64_t m, int64_t n, int64_t k,
                             const double* A, int64_t lda, const double* B, int64_t ldb, int p, int32_t* Cs,
                             emu_stream_t stream) {
  emu_status_t s = gemm_common(h, layout, m, n, k, A, lda, B, ldb, Cs, layout == EMU_ROW_MAJOR ? n : m,
                               EMU_SCHEME_I_F8, p);
  if (s != EMU_OK) return s;
  if (k > host_chunk_len_F8(p)) return EMU_ERR_UNSUPPORTED;
  if (layout != EMU_ROW_MAJOR) return EMU_ERR_UNSUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  View v;
  normalize(layout, m, n, A, lda, B, ldb, &v);
  if (v.M == 0 || v.N == 0) return EMU_OK;
  if (k == 0) return cuda_err(cudaMemsetAsync(Cs, 0, sizeof(int32_t) * p * v.M * v.N, st));
  return run_scheme_I<double>(h, v, k, p, 1.0, 0.0, nullptr, 0, OUT_PARTIALS, Cs, st, nullptr, true);
}

emu_status_t emu_residues_II(emu_handle_t h, emu_layout_t layout, int64_t m, int64_t n, int64_t k,
                             const double* A, int64_t lda, const double* B, int64_t ldb, int nm, uint8_t* R,
                             emu_stream_t stream) {
  emu_status_t s = gemm_common(h, layout, m, n, k, A, lda, B, ldb, R, layout == EMU_ROW_MAJOR ? n : m,
                               EMU_SCHEME_II, nm);
  if (s != EMU_OK) return s;
  if (layout != EMU_ROW_MAJOR) return EMU_ERR_UNSUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  View v;
  normalize(layout, m, n, A, lda, B, ldb, &v);
  if (v.M == 0 || v.N == 0) return EMU_OK;
  if (k == 0) return cuda_err(cudaMemsetAsync(R, 0, static_cast<size_t>(nm) * v.M * v.N, st));
  return run_scheme_II<double>(h, v, k, nm, 1, 1.0, 0.0, 0.0, 0.0, nullptr, 0, II_RESIDUES, R, st);
}

}  // extern "C"
