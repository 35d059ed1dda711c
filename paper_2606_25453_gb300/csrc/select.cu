// select.cu -- learned slice-count selector for Scheme I (auto precision).
//
// The paper picks p by hand and notes that it lacks an automatic precision
// choice (Sec. VII).  This file adds one: per-product features (exponent
// deficit histograms of sampled rows of A and columns of B, log2 k and the
// requested tolerance), a 66-64-64-8 MLP with hand-written FP32 forward,
// backward and Adam kernels, a double-double probe of sampled output entries
// that judges a prediction, and emu_dgemm_auto, which escalates p when the
// probe finds the tolerance missed.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "emu_handle.h"
#include "emu_internal.h"

namespace emu {

namespace {

constexpr int kIn = EMU_SEL_IN, kHid = EMU_SEL_HID, kOut = EMU_SEL_OUT;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kHid * kIn, kOffW2 = kOffB1 + kHid, kOffB2 = kOffW2 + kHid * kHid,
              kOffW3 = kOffB2 + kHid, kOffB3 = kOffW3 + kOut * kHid, kNParam = kOffB3 + kOut;
static_assert(kNParam == EMU_SEL_NPARAM, "parameter count");

struct SelState {
  float* params = nullptr;  // device, loaded weights (Scheme I: classes p = 3..10)
  bool loaded = false;
  float* params_II = nullptr;  // Scheme II, norm scaling: classes N = 6, 8, .., 20
  bool loaded_II = false;
  // auto-precision buffers, grown on demand: device [feat 128 | prob 8 |
  // probe idx | probe results], and a pinned host copy of the parts read
  // back, so that each decision costs one device-to-host copy
  uint8_t* dev = nullptr;
  size_t dev_bytes = 0;
  uint8_t* host = nullptr;
  size_t host_bytes = 0;
  // side stream for the probe's reference sums (they depend on A and B
  // only, so they run beside the feature pass and the product)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_probe = nullptr;
};
SelState* sel_of(emu_handle_s* h) {
  if (!h->selector) h->selector = new SelState();
  return static_cast<SelState*>(h->selector);
}

// ---------------------------------------------------------------- features
// Exponent of |x| from its bits: frexp exponent (E with |x| in [2^(E-1), 2^E)).
__device__ __forceinline__ int exp_bits(uint64_t ab) { return frexp_exp_bits(ab); }

// One block per sampled vector: 32-bin histogram of the exponent deficit
// d = E_vec - e(x) in bins of 3 exponents (bin = min(d / 3, 31); x == 0 ->
// bin 31), added to hist (uint32[32]).  E_vec, the exponent of the vector's
// largest magnitude, is found by the block first (the vector is then read
// a second time, from L2), so that no pass over the whole of A and B is
// needed for 64 sampled vectors.
// One launch serves both operands: blocks [0, nblk_a) sample A (histogram
// hist[0..31]), the rest sample B (hist[32..63]).
struct FeatOperand {
  const double* X;
  int64_t ld;
  bool kcontig;
  int64_t rows, stride;
};
__global__ void feat_hist_kernel(FeatOperand oa, FeatOperand ob, int nblk_a, int64_t k,
                                 unsigned int* __restrict__ hist_all) {
  __shared__ unsigned int sh[32];
  __shared__ unsigned long long shmax;
  if (threadIdx.x < 32) sh[threadIdx.x] = 0;
  if (threadIdx.x == 0) shmax = 0;
  __syncthreads();
  const bool is_a = static_cast<int>(blockIdx.x) < nblk_a;
  const FeatOperand& op = is_a ? oa : ob;
  const double* __restrict__ X = op.X;
  const int64_t ld = op.ld, rows = op.rows;
  const bool kcontig = op.kcontig;
  unsigned int* __restrict__ hist = hist_all + (is_a ? 0 : 32);
  int64_t r = static_cast<int64_t>(is_a ? blockIdx.x : blockIdx.x - nblk_a) * op.stride;
  if (r < rows) {
    unsigned long long mx = 0;  // largest |x| bit pattern (NaN > inf > finite)
    for (int64_t h = threadIdx.x; h < k; h += blockDim.x) {
      const unsigned long long ab = dbits(__ldg(kcontig ? X + r * ld + h : X + h * ld + r)) & 0x7FFFFFFFFFFFFFFFull;
      mx = ab > mx ? ab : mx;
    }
    for (int o = 16; o; o >>= 1) {
      const unsigned long long other = __shfl_xor_sync(0xffffffffu, mx, o);
      mx = other > mx ? other : mx;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(&shmax, mx);
  }
  __syncthreads();
  if (r < rows) {
    const uint64_t mb = shmax;
    int E = mb >= 0x7FF0000000000000ull ? 0 : exp_bits(mb);
    for (int64_t h = threadIdx.x; h < k; h += blockDim.x) {
      uint64_t ab = dbits(__ldg(kcontig ? X + r * ld + h : X + h * ld + r)) & 0x7FFFFFFFFFFFFFFFull;
      int bin = 31;
      if (ab != 0 && ab < 0x7FF0000000000000ull) {
        int d = E - exp_bits(ab);
        bin = d < 0 ? 0 : (d / 3 > 31 ? 31 : d / 3);
      }
      atomicAdd(&sh[bin], 1u);
    }
  }
  __syncthreads();
  if (threadIdx.x < 32 && sh[threadIdx.x]) atomicAdd(&hist[threadIdx.x], sh[threadIdx.x]);
}

__global__ void feat_finalize_kernel(const unsigned int* __restrict__ hist, double log2k, double ltol,
                                     float* __restrict__ feat) {
  int t = threadIdx.x;
  __shared__ float tot[2];
  if (t < 2) {
    unsigned int s = 0;
    for (int i = 0; i < 32; ++i) s += hist[t * 32 + i];
    tot[t] = s ? static_cast<float>(s) : 1.0f;
  }
  __syncthreads();
  if (t < 64) feat[t] = static_cast<float>(hist[t]) / tot[t / 32];
  if (t == 64) feat[64] = static_cast<float>(log2k / 16.0);
  if (t == 65) feat[65] = static_cast<float>(ltol / 16.0);
}

// ---------------------------------------------------------------- MLP
// One block of 64 threads per sample.  act (optional): [h1 | h2] per sample.
__global__ void mlp_forward_kernel(const float* __restrict__ prm, const float* __restrict__ X, int64_t batch,
                                   float* __restrict__ P, float* __restrict__ act) {
  __shared__ float x[kIn], h1[kHid], h2[kHid], z[kOut];
  const int64_t b = blockIdx.x;
  const int j = threadIdx.x;
  if (b >= batch) return;
  for (int i = j; i < kIn; i += blockDim.x) x[i] = X[b * kIn + i];
  __syncthreads();
  float s = prm[kOffB1 + j];
  for (int i = 0; i < kIn; ++i) s = fmaf(prm[kOffW1 + j * kIn + i], x[i], s);
  h1[j] = s > 0.f ? s : 0.f;
  __syncthreads();
  s = prm[kOffB2 + j];
  for (int i = 0; i < kHid; ++i) s = fmaf(prm[kOffW2 + j * kHid + i], h1[i], s);
  h2[j] = s > 0.f ? s : 0.f;
  __syncthreads();
  if (j < kOut) {
    float t = prm[kOffB3 + j];
    for (int i = 0; i < kHid; ++i) t = fmaf(prm[kOffW3 + j * kHid + i], h2[i], t);
    z[j] = t;
  }
  __syncthreads();
  if (j < kOut) {
    float mx = z[0];
    for (int o = 1; o < kOut; ++o) mx = fmaxf(mx, z[o]);
    float den = 0.f;
    for (int o = 0; o < kOut; ++o) den += expf(z[o] - mx);
    P[b * kOut + j] = expf(z[j] - mx) / den;
  }
  if (act) {
    act[b * 2 * kHid + j] = h1[j];
    act[b * 2 * kHid + kHid + j] = h2[j];
  }
}

// Mean cross-entropy backward.  Each block takes `per` samples, accumulates
// the parameter gradient in shared memory and adds it to grad once.
__global__ void mlp_backward_kernel(const float* __restrict__ prm, const float* __restrict__ X,
                                    const float* __restrict__ act, const float* __restrict__ P,
                                    const int32_t* __restrict__ y, int64_t batch, int per, float* __restrict__ grad,
                                    float* __restrict__ loss) {
  extern __shared__ float g[];  // kNParam floats
  __shared__ float dz[kOut], dh2[kHid], dh1[kHid];
  const int j = threadIdx.x;  // 64 threads
  for (int i = j; i < kNParam; i += blockDim.x) g[i] = 0.f;
  __syncthreads();
  const float inv = 1.0f / static_cast<float>(batch);
  float lsum = 0.f;
  for (int q = 0; q < per; ++q) {
    int64_t b = static_cast<int64_t>(blockIdx.x) * per + q;
    if (b >= batch) break;
    const float* x = X + b * kIn;
    const float* h1 = act + b * 2 * kHid;
    const float* h2 = h1 + kHid;
    const int lab = y[b];
    if (j < kOut) dz[j] = (P[b * kOut + j] - (j == lab ? 1.f : 0.f)) * inv;
    if (j == 0) lsum += -logf(fmaxf(P[b * kOut + lab], 1e-30f));
    __syncthreads();
    // layer 3
    for (int o = 0; o < kOut; ++o) g[kOffW3 + o * kHid + j] += dz[o] * h2[j];
    if (j < kOut) g[kOffB3 + j] += dz[j];
    float s = 0.f;
    for (int o = 0; o < kOut; ++o) s = fmaf(prm[kOffW3 + o * kHid + j], dz[o], s);
    dh2[j] = h2[j] > 0.f ? s : 0.f;
    __syncthreads();
    // layer 2 (thread j owns row j of W2)
    for (int i = 0; i < kHid; ++i) g[kOffW2 + j * kHid + i] += dh2[j] * h1[i];
    g[kOffB2 + j] += dh2[j];
    s = 0.f;
    for (int o = 0; o < kHid; ++o) s = fmaf(prm[kOffW2 + o * kHid + j], dh2[o], s);
    dh1[j] = h1[j] > 0.f ? s : 0.f;
    __syncthreads();
    // layer 1 (thread j owns row j of W1)
    for (int i = 0; i < kIn; ++i) g[kOffW1 + j * kIn + i] += dh1[j] * x[i];
    g[kOffB1 + j] += dh1[j];
    __syncthreads();
  }
  for (int i = j; i < kNParam; i += blockDim.x)
    if (g[i] != 0.f) atomicAdd(&grad[i], g[i]);
  if (j == 0 && lsum != 0.f) atomicAdd(loss, lsum * inv);
}

__global__ void adam_kernel(float* __restrict__ prm, const float* __restrict__ grad, float* __restrict__ m,
                            float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float c1, float c2) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float gi = grad[i];
  float mi = b1 * m[i] + (1.f - b1) * gi;
  float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  prm[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// ---------------------------------------------------------------- probe
struct DD {
  double hi, lo;
};
__device__ __forceinline__ DD dd_add(DD a, DD b) {
  double s = __dadd_rn(a.hi, b.hi);
  double z = __dsub_rn(s, a.hi);
  double e = __dadd_rn(__dsub_rn(a.hi, __dsub_rn(s, z)), __dsub_rn(b.hi, z));
  e = __dadd_rn(e, __dadd_rn(a.lo, b.lo));
  double t = __dadd_rn(s, e);
  return {t, __dsub_rn(e, __dsub_rn(t, s))};
}

// One block of kProbeThreads per sampled entry (i, j): compensated dot
// product (TwoProduct by fma, TwoSum accumulation) per thread over a strided
// share of K, threads combined by double-double adds (warp shuffles, then
// the warps' partial results through shared memory).  A block per entry
// keeps many independent loads in flight: one warp walking all of K waited
// on one strided load per step.
constexpr int kProbeThreads = 256;
__global__ void __launch_bounds__(kProbeThreads) probe_dd_kernel(const double* __restrict__ A, int64_t lda,
                                                                bool a_kcontig, const double* __restrict__ B,
                                                                int64_t ldb, bool b_kcontig, int64_t k, int count,
                                                                const int32_t* __restrict__ idx,
                                                                double* __restrict__ ref, double* __restrict__ absab) {
  __shared__ double sh[3][kProbeThreads / 32];
  const int w = blockIdx.x, lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  if (w >= count) return;
  const int64_t i = idx[2 * w], j = idx[2 * w + 1];
  DD acc{0.0, 0.0};
  double ab = 0.0;
  for (int64_t h = threadIdx.x; h < k; h += kProbeThreads) {
    const double a = a_kcontig ? A[i * lda + h] : A[h * lda + i];
    const double b = b_kcontig ? B[j * ldb + h] : B[h * ldb + j];
    const double p = __dmul_rn(a, b);
    const double e = __fma_rn(a, b, -p);
    acc = dd_add(acc, DD{p, e});
    ab = __fma_rn(fabs(a), fabs(b), ab);
  }
  for (int o = 16; o; o >>= 1) {
    DD other{__shfl_xor_sync(0xffffffffu, acc.hi, o), __shfl_xor_sync(0xffffffffu, acc.lo, o)};
    acc = dd_add(acc, other);
    ab = __dadd_rn(ab, __shfl_xor_sync(0xffffffffu, ab, o));
  }
  if (lane == 0) {
    sh[0][wp] = acc.hi;
    sh[1][wp] = acc.lo;
    sh[2][wp] = ab;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    DD t{sh[0][0], sh[1][0]};
    double tab = sh[2][0];
    for (int q = 1; q < kProbeThreads / 32; ++q) {
      t = dd_add(t, DD{sh[0][q], sh[1][q]});
      tab = __dadd_rn(tab, sh[2][q]);
    }
    ref[2 * w] = t.hi;
    ref[2 * w + 1] = t.lo;
    absab[w] = tab;
  }
}

// idx pairs (i, j) -> (j, i), for gathering entries of a column-major C.
__global__ void swap_pairs_kernel(const int32_t* __restrict__ idx, int count, int32_t* __restrict__ out) {
  int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w < count) {
    out[2 * w] = idx[2 * w + 1];
    out[2 * w + 1] = idx[2 * w];
  }
}

__global__ void gather_kernel(const double* __restrict__ C, int64_t ldc, int count, const int32_t* __restrict__ idx,
                              double* __restrict__ out) {
  int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w < count) out[w] = C[static_cast<int64_t>(idx[2 * w]) * ldc + idx[2 * w + 1]];
}

}  // namespace

void selector_release(emu_handle_s* h) {
  auto* s = static_cast<SelState*>(h->selector);
  if (!s) return;
  if (s->params) cudaFree(s->params);
  if (s->params_II) cudaFree(s->params_II);
  if (s->dev) cudaFree(s->dev);
  if (s->host) cudaFreeHost(s->host);
  if (s->side) cudaStreamDestroy(s->side);
  if (s->ev_fork) cudaEventDestroy(s->ev_fork);
  if (s->ev_probe) cudaEventDestroy(s->ev_probe);
  delete s;
  h->selector = nullptr;
}

}  // namespace emu

using namespace emu;

namespace {

// Features of one product into feat (device float[66]); needs 8*(m+n)+256
// bytes of scratch (maxbits + histogram).
emu_status_t features_impl(emu_handle_s* h, const View& v, int64_t k, double tol, int64_t sample, float* feat,
                           uint8_t* scratch, cudaStream_t st) {
  auto* hist = reinterpret_cast<unsigned int*>(scratch);
  cudaMemsetAsync(hist, 0, 64 * sizeof(unsigned int), st);
  int64_t sa = sample > 0 ? std::max<int64_t>(1, v.M / sample) : 1;
  int64_t sb = sample > 0 ? std::max<int64_t>(1, v.N / sample) : 1;
  int64_t na = (v.M + sa - 1) / sa, nb = (v.N + sb - 1) / sb;
  if (sample > 0) {
    na = std::min<int64_t>(na, sample);
    nb = std::min<int64_t>(nb, sample);
  }
  const FeatOperand oa{static_cast<const double*>(v.A), v.ldA, v.a_kcontig, v.M, sa};
  const FeatOperand ob{static_cast<const double*>(v.B), v.ldB, v.b_kcontig, v.N, sb};
  feat_hist_kernel<<<static_cast<unsigned>(na + nb), 256, 0, st>>>(oa, ob, static_cast<int>(na), k, hist);
  feat_finalize_kernel<<<1, 96, 0, st>>>(hist, std::log2(static_cast<double>(k)), -std::log10(tol), feat);
  return cudaGetLastError() == cudaSuccess ? EMU_OK : EMU_ERR_CUDA;
}

size_t feat_scratch(const View&) { return 512; }

bool valid_layout(emu_layout_t l) { return l == EMU_ROW_MAJOR || l == EMU_COL_MAJOR; }

// Bound-based p: smallest p in [3, 10] with 2^(-8p+3) * 2^spread * k <= tol,
// spread = the upper edge of the largest exponent-deficit bin seen.
// Scheme II with norm scaling: a' = trunc(a 2^(h - e_i)) errs by less than
// 2^(e_i - h) and e_i exceeds the frexp exponent of an entry by at most the
// deficit d against the row maximum plus ceil(log2(k) / 2), so every term
// of the product errs by at most 2^(-h + d + ceil(log2(k)/2) + 3) of its
// magnitude.  Smallest N in 6, 8, .., 20 meeting tol with d = spread (20 if
// none does).  A heuristic fallback, like the Scheme I bound.
int bound_nm_from_hist(const float* f, int64_t k, double tol) {
  int spread = 0;
  for (int i = 0; i < 64; ++i)
    if (f[i] > 0.f) spread = std::max(spread, 3 * (i % 32) + 2);
  int half_lk = 0;
  while ((int64_t{1} << (2 * half_lk)) < k) ++half_lk;  // ceil(log2(k) / 2)
  for (int nm = EMU_SEL_NM0; nm <= EMU_NM_MAX; nm += 2) {
    int hA, hB;
    host_norm_halves_II(nm, &hA, &hB);
    if (std::ldexp(1.0, -hA + spread + half_lk + 3) <= tol) return nm;
  }
  return EMU_NM_MAX;
}

int bound_p_from_hist(const float* f, int64_t k, double tol) {
  int spread = 0;
  for (int i = 0; i < 64; ++i)
    if (f[i] > 0.f) spread = std::max(spread, 3 * (i % 32) + 2);
  for (int p = 3; p <= 10; ++p)
    if (std::ldexp(1.0, -8 * p + 3 + spread) * static_cast<double>(k) <= tol) return p;
  return 10;
}

// Bound-based choice (host), shared by emu_bound_p and emu_bound_nm.
emu_status_t bound_impl(emu_handle_s* h, emu_layout_t layout, int64_t m, int64_t n, int64_t k, const double* A,
                        int64_t lda, const double* B, int64_t ldb, double tol, int* out, emu_stream_t stream,
                        bool scheme_II) {
  if (!out || !h) return EMU_ERR_INVALID_ARG;
  if ((layout != EMU_ROW_MAJOR && layout != EMU_COL_MAJOR) || m < 1 || n < 1 || k < 1 || !A || !B || !(tol > 0.0))
    return EMU_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  View v;
  normalize(layout, m, n, A, lda, B, ldb, &v);
  uint8_t* ws = nullptr;
  const size_t need = feat_scratch(v) + 512;
  emu_status_t s = handle_workspace(h, need, st, &ws);
  if (s != EMU_OK) return s;
  float* feat = reinterpret_cast<float*>(ws + feat_scratch(v));
  s = features_impl(h, v, k, tol, 64, feat, ws, st);
  if (s != EMU_OK) return s;
  float f[kIn];
  if (cudaMemcpyAsync(f, feat, sizeof(f), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return EMU_ERR_CUDA;
  *out = scheme_II ? bound_nm_from_hist(f, k, tol) : bound_p_from_hist(f, k, tol);
  return EMU_OK;
}

}  // namespace

extern "C" {

emu_status_t emu_sel_features(emu_handle_t h, emu_layout_t layout, int64_t m, int64_t n, int64_t k, const double* A,
                              int64_t lda, const double* B, int64_t ldb, double tol, int64_t sample, float* feat,
                              emu_stream_t stream) {
  if (!h || !feat || !A || !B || m < 1 || n < 1 || k < 1 || !(tol > 0.0) || !valid_layout(layout))
    return EMU_ERR_INVALID_ARG;
  if (!check_lds(layout, m, n, k, lda, ldb, layout == EMU_ROW_MAJOR ? n : m)) return EMU_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  View v;
  normalize(layout, m, n, A, lda, B, ldb, &v);
  uint8_t* ws = nullptr;
  emu_status_t s = handle_workspace(h, feat_scratch(v), st, &ws);
  if (s != EMU_OK) return s;
  return features_impl(h, v, k, tol, sample, feat, ws, st);
}

emu_status_t emu_sel_forward(emu_handle_t h, int64_t batch, const float* prm, const float* X, float* P, float* act,
                             emu_stream_t stream) {
  if (!h || !prm || !X || !P || batch < 0) return EMU_ERR_INVALID_ARG;
  if (batch == 0) return EMU_OK;
  if (batch > INT32_MAX) return EMU_ERR_UNSUPPORTED;
  cudaSetDevice(h->device);
  mlp_forward_kernel<<<static_cast<unsigned>(batch), kHid, 0, static_cast<cudaStream_t>(stream)>>>(prm, X, batch, P,
                                                                                                    act);
  return cudaGetLastError() == cudaSuccess ? EMU_OK : EMU_ERR_CUDA;
}

emu_status_t emu_sel_backward(emu_handle_t h, int64_t batch, const float* prm, const float* X, const float* act,
                              const float* P, const int32_t* y, float* grad, float* loss, emu_stream_t stream) {
  if (!h || !prm || !X || !act || !P || !y || !grad || !loss || batch < 1) return EMU_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int per = 32;
  const int smem = kNParam * static_cast<int>(sizeof(float));
  if (cudaFuncSetAttribute(mlp_backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
    return EMU_ERR_CUDA;
  cudaMemsetAsync(grad, 0, sizeof(float) * kNParam, st);
  cudaMemsetAsync(loss, 0, sizeof(float), st);
  unsigned blocks = static_cast<unsigned>((batch + per - 1) / per);
  mlp_backward_kernel<<<blocks, kHid, smem, st>>>(prm, X, act, P, y, batch, per, grad, loss);
  return cudaGetLastError() == cudaSuccess ? EMU_OK : EMU_ERR_CUDA;
}

emu_status_t emu_sel_adam(emu_handle_t h, float* prm, const float* grad, float* m, float* v, int step, float lr,
                          float b1, float b2, float eps, emu_stream_t stream) {
  if (!h || !prm || !grad || !m || !v || step < 1) return EMU_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  float c1 = 1.f - std::pow(b1, static_cast<float>(step)), c2 = 1.f - std::pow(b2, static_cast<float>(step));
  adam_kernel<<<(kNParam + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(prm, grad, m, v, kNParam, lr, b1,
                                                                                      b2, eps, c1, c2);
  return cudaGetLastError() == cudaSuccess ? EMU_OK : EMU_ERR_CUDA;
}

emu_status_t emu_sel_load(emu_handle_t h, const float* params) {
  if (!h || !params) return EMU_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  SelState* s = sel_of(h);
  if (!s->params && cudaMalloc(&s->params, sizeof(float) * kNParam) != cudaSuccess) return EMU_ERR_ALLOC;
  if (cudaMemcpy(s->params, params, sizeof(float) * kNParam, cudaMemcpyHostToDevice) != cudaSuccess)
    return EMU_ERR_CUDA;
  s->loaded = true;
  return EMU_OK;
}

emu_status_t emu_sel_load_II(emu_handle_t h, const float* params) {
  if (!h || !params) return EMU_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  SelState* s = sel_of(h);
  if (!s->params_II && cudaMalloc(&s->params_II, sizeof(float) * kNParam) != cudaSuccess) return EMU_ERR_ALLOC;
  if (cudaMemcpy(s->params_II, params, sizeof(float) * kNParam, cudaMemcpyHostToDevice) != cudaSuccess)
    return EMU_ERR_CUDA;
  s->loaded_II = true;
  return EMU_OK;
}

emu_status_t emu_probe_dd(emu_handle_t h, emu_layout_t layout, int64_t m, int64_t n, int64_t k, const double* A,
                          int64_t lda, const double* B, int64_t ldb, int count, const int32_t* idx, double* ref,
                          double* absab, emu_stream_t stream) {
  if (!h || !A || !B || !idx || !ref || !absab || count < 0 || m < 1 || n < 1 || k < 1 || !valid_layout(layout))
    return EMU_ERR_INVALID_ARG;
  if (!check_lds(layout, m, n, k, lda, ldb, layout == EMU_ROW_MAJOR ? n : m)) return EMU_ERR_INVALID_ARG;
  if (count == 0) return EMU_OK;
  cudaSetDevice(h->device);
  // entries are given in the caller's (i, j) of C; the kernel reads A rows
  // and B columns directly in the caller's layout
  bool a_k = layout == EMU_ROW_MAJOR, b_k = layout != EMU_ROW_MAJOR;
  probe_dd_kernel<<<count, kProbeThreads, 0, static_cast<cudaStream_t>(stream)>>>(A, lda, a_k, B, ldb, b_k, k,
                                                                                 count, idx, ref, absab);
  return cudaGetLastError() == cudaSuccess ? EMU_OK : EMU_ERR_CUDA;
}

emu_status_t emu_bound_p(emu_handle_t h, emu_layout_t layout, int64_t m, int64_t n, int64_t k, const double* A,
                         int64_t lda, const double* B, int64_t ldb, double tol, int* p_out, emu_stream_t stream) {
  return bound_impl(h, layout, m, n, k, A, lda, B, ldb, tol, p_out, stream, false);
}

emu_status_t emu_bound_nm(emu_handle_t h, emu_layout_t layout, int64_t m, int64_t n, int64_t k, const double* A,
                          int64_t lda, const double* B, int64_t ldb, double tol, int* nm_out, emu_stream_t stream) {
  return bound_impl(h, layout, m, n, k, A, lda, B, ldb, tol, nm_out, stream, true);
}

}  // extern "C"

namespace {
// Shared by the Scheme I (p) and Scheme II (N moduli, norm scaling) auto
// entry points: selector class -> value, probe, escalation.
emu_status_t auto_impl(emu_handle_t h, emu_layout_t layout, int64_t m, int64_t n, int64_t k, double alpha,
                       const double* A, int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc,
                       double tol, int probe, int* p_used, emu_stream_t stream, bool scheme_II) {
  if (!h || !p_used || !A || !B || !C || m < 1 || n < 1 || k < 1 || !(tol > 0.0) || probe < 0 || !valid_layout(layout))
    return EMU_ERR_INVALID_ARG;
  if (!check_lds(layout, m, n, k, lda, ldb, ldc)) return EMU_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  SelState* ss = sel_of(h);
  View v;
  normalize(layout, m, n, A, lda, B, ldb, &v);
  // selector buffers: features and probabilities (136 floats), then the
  // probe's indices, its results [ref (hi, lo) | sum |a||b| | C entry], and
  // the swapped index pairs of a column-major gather
  const int pc = std::max(probe, 1);
  const size_t off_idx = 1024, off_res = off_idx + (8 * static_cast<size_t>(pc) + 255) / 256 * 256;
  const size_t dev_need = off_res + 40 * static_cast<size_t>(pc);
  const size_t host_need = std::max<size_t>(1024, 32 * static_cast<size_t>(pc));
  if (dev_need > ss->dev_bytes) {
    if (ss->dev) cudaFree(ss->dev);
    ss->dev = nullptr;
    ss->dev_bytes = 0;
    if (cudaMalloc(&ss->dev, dev_need) != cudaSuccess) {
      cudaGetLastError();
      return EMU_ERR_ALLOC;
    }
    ss->dev_bytes = dev_need;
  }
  if (host_need > ss->host_bytes) {
    if (ss->host) cudaFreeHost(ss->host);
    ss->host = nullptr;
    ss->host_bytes = 0;
    if (cudaMallocHost(&ss->host, host_need) != cudaSuccess) {
      cudaGetLastError();
      return EMU_ERR_ALLOC;
    }
    ss->host_bytes = host_need;
  }
  float* feat = reinterpret_cast<float*>(ss->dev);
  float* prob = feat + 128;
  // probe entries: a deterministic spread over C (caller's coordinates),
  // uploaded once for every attempt (row-major view: (i, j); column-major C:
  // element (i, j) sits at row j, column i of the row-major view); their
  // double-double reference sums depend on A and B only, so they run on a
  // side stream beside the feature pass and the product
  auto* d_idx = reinterpret_cast<int32_t*>(ss->dev + off_idx);
  auto* d_ref = reinterpret_cast<double*>(ss->dev + off_res);
  auto* d_ab = d_ref + 2 * pc;
  auto* d_c = d_ab + pc;
  auto* d_sw = reinterpret_cast<int32_t*>(d_c + pc);  // gather indices for column-major C
  if (probe > 0) {
    if (!ss->side && (cudaStreamCreateWithFlags(&ss->side, cudaStreamNonBlocking) != cudaSuccess ||
                      cudaEventCreateWithFlags(&ss->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
                      cudaEventCreateWithFlags(&ss->ev_probe, cudaEventDisableTiming) != cudaSuccess))
      return EMU_ERR_CUDA;
    auto* hidx = reinterpret_cast<int32_t*>(ss->host);
    uint64_t x = 0x9E3779B97F4A7C15ull ^ static_cast<uint64_t>(m * 1315423911u + n * 2654435761u + k);
    for (int q = 0; q < probe; ++q) {
      x ^= x << 13;
      x ^= x >> 7;
      x ^= x << 17;
      hidx[2 * q] = static_cast<int32_t>(x % static_cast<uint64_t>(m));
      x ^= x << 13;
      x ^= x >> 7;
      x ^= x << 17;
      hidx[2 * q + 1] = static_cast<int32_t>(x % static_cast<uint64_t>(n));
    }
    // (the host buffer is next written by the features' copy, which the
    // stream orders after this one)
    if (cudaMemcpyAsync(d_idx, hidx, 8 * static_cast<size_t>(probe), cudaMemcpyHostToDevice, st) != cudaSuccess)
      return EMU_ERR_CUDA;
    if (layout != EMU_ROW_MAJOR) swap_pairs_kernel<<<(probe + 127) / 128, 128, 0, st>>>(d_idx, probe, d_sw);
    if (cudaEventRecord(ss->ev_fork, st) != cudaSuccess || cudaStreamWaitEvent(ss->side, ss->ev_fork, 0) != cudaSuccess)
      return EMU_ERR_CUDA;
    emu_status_t s = emu_probe_dd(h, layout, m, n, k, A, lda, B, ldb, probe, d_idx, d_ref, d_ab, ss->side);
    if (s != EMU_OK) return s;
    if (cudaEventRecord(ss->ev_probe, ss->side) != cudaSuccess) return EMU_ERR_CUDA;
  }
  {  // the feature scan needs scratch for the row / column maxima and histograms
    uint8_t* ws = nullptr;
    emu_status_t s = handle_workspace(h, feat_scratch(v), st, &ws);
    if (s != EMU_OK) return s;
    s = features_impl(h, v, k, tol, 64, feat, ws, st);
    if (s != EMU_OK) return s;
  }
  const bool loaded = scheme_II ? ss->loaded_II : ss->loaded;
  if (loaded) mlp_forward_kernel<<<1, kHid, 0, st>>>(scheme_II ? ss->params_II : ss->params, feat, 1, prob, nullptr);
  // one copy back: features and (if a network is loaded) probabilities
  if (cudaMemcpyAsync(ss->host, feat, sizeof(float) * (128 + kOut), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return EMU_ERR_CUDA;
  const float* f = reinterpret_cast<const float*>(ss->host);
  const float* pr = f + 128;
  // value of class c and the largest value: p = 3 + c up to EMU_P_MAX, or
  // N = 6 + 2c up to EMU_NM_MAX
  const int top = scheme_II ? EMU_NM_MAX : EMU_P_MAX;
  const int step = scheme_II ? 2 : 1;
  const int base_v = scheme_II ? EMU_SEL_NM0 : EMU_SEL_P0;
  const int pb = scheme_II ? bound_nm_from_hist(f, k, tol) : bound_p_from_hist(f, k, tol);
  int p = pb;
  if (loaded) {  // smallest class whose cumulative predicted probability reaches 0.8
    float c = 0.f;
    int cls = kOut - 1;
    for (int o = 0; o < kOut; ++o) {
      c += pr[o];
      if (c >= 0.8f) {
        cls = o;
        break;
      }
    }
    // the top class is open-ended ("10 or more" / "20"): go to the largest value at once
    p = cls == kOut - 1 ? top : base_v + step * cls;
  }
  for (int attempt = 0; attempt < 3; ++attempt) {
    emu_status_t s = emu_dgemm(h, layout, m, n, k, alpha, A, lda, B, ldb, 0.0, C, ldc,
                               scheme_II ? EMU_SCHEME_II_NORM : EMU_SCHEME_I, p, stream);
    if (s != EMU_OK) return s;
    *p_used = p;
    if (probe == 0) return EMU_OK;
    if (attempt == 0 && cudaStreamWaitEvent(st, ss->ev_probe, 0) != cudaSuccess) return EMU_ERR_CUDA;
    gather_kernel<<<(probe + 127) / 128, 128, 0, st>>>(C, ldc, probe, layout == EMU_ROW_MAJOR ? d_idx : d_sw, d_c);
    // one copy back: [ref | ab | C entries]
    if (cudaMemcpyAsync(ss->host, d_ref, 32 * static_cast<size_t>(probe), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return EMU_ERR_CUDA;
    const double* ref = reinterpret_cast<const double*>(ss->host);
    const double* ab = ref + 2 * probe;
    const double* cv = ab + probe;
    double worst = 0.0;
    for (int q = 0; q < probe; ++q) {
      double d = std::fabs((cv[q] / alpha - ref[2 * q]) - ref[2 * q + 1]);
      double e = ab[q] > 0.0 ? d / ab[q] : (d > 0.0 ? INFINITY : 0.0);
      worst = std::max(worst, e);
    }
    if (worst <= tol) return EMU_OK;
    if (p >= top) return EMU_ERR_TOL_NOT_MET;
    // a miss at the top class goes straight to the largest value
    p = (attempt == 0 && p < base_v + step * (kOut - 1)) ? std::max(p + step, pb) : top;
    p = std::min(p, top);
  }
  return EMU_ERR_TOL_NOT_MET;
}
}  // namespace

extern "C" {

emu_status_t emu_dgemm_auto(emu_handle_t h, emu_layout_t layout, int64_t m, int64_t n, int64_t k, double alpha,
                            const double* A, int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc,
                            double tol, int probe, int* p_used, emu_stream_t stream) {
  return auto_impl(h, layout, m, n, k, alpha, A, lda, B, ldb, C, ldc, tol, probe, p_used, stream, false);
}

emu_status_t emu_dgemm_auto_II(emu_handle_t h, emu_layout_t layout, int64_t m, int64_t n, int64_t k, double alpha,
                               const double* A, int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc,
                               double tol, int probe, int* nm_used, emu_stream_t stream) {
  return auto_impl(h, layout, m, n, k, alpha, A, lda, B, ldb, C, ldc, tol, probe, nm_used, stream, true);
}



}  // extern "C"
