// Batched BLAS-1 and the per-right-hand-side GMRES bookkeeping.
//
// Reductions are deterministic and independent of the batch: every rhs is
// reduced over the same fixed partition of its vector (stage 1: one partial
// per CTA-chunk, stage 2: one CTA sums the partials in a fixed order), so a
// right-hand side gives bit-identical results alone or inside a batch.
#include "common.cuh"
#include "kernels.h"

#include <stdexcept>
#include <unordered_map>

#include <cstdio>
#include <atomic>
#include <mutex>

namespace {

constexpr int RT = 256;         // threads per reduction CTA
constexpr int MAXCHUNKS = 512;  // partials per rhs (and per dot in a multidot)

// scratch for the partials, one buffer per stream (reductions issued on different streams, as by
// the serving workers of several hierarchies, never share scratch), grown on demand
// (library-owned device memory).  A buffer that was replaced is kept until the library is
// unloaded, because captured CUDA graphs may still refer to it.
struct PartialBuf {
  double* p = nullptr;
  size_t cap = 0;
};
std::mutex g_partials_mu;
std::unordered_map<cudaStream_t, PartialBuf> g_partials;

double* partials(size_t count, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_partials_mu);
  PartialBuf& b = g_partials[st];
  if (count > b.cap) {
    const size_t cap = count < (1u << 17) ? (1u << 17) : count;
    double* p = nullptr;
    if (cudaMalloc(&p, cap * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      throw std::runtime_error("out of device memory for reduction partials");
    }
    b.p = p;
    b.cap = cap;
  }
  return b.p;
}

int nchunks(size_t len) {
  size_t c = (len + 4 * RT - 1) / (4 * RT);
  if (c < 1) c = 1;
  if (c > MAXCHUNKS) c = MAXCHUNKS;
  return (int)c;
}

__device__ double warp_sum(double v) {
  for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// sum `cnt` doubles per thread over the CTA (cnt <= 8); thread 0 gets the result
__device__ void cta_sum(double* v, int cnt, double* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 0; k < cnt; ++k) v[k] = warp_sum(v[k]);
  if (lane == 0)
    for (int k = 0; k < cnt; ++k) sh[warp * 8 + k] = v[k];
  __syncthreads();
  if (threadIdx.x == 0)
    for (int k = 0; k < cnt; ++k) {
      double s = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w * 8 + k];
      v[k] = s;
    }
  __syncthreads();
}

// chunk [lo, hi) of a vector of length len split into nc chunks
__device__ void chunk_range(size_t len, int nc, int c, size_t& lo, size_t& hi) {
  const size_t per = (len + nc - 1) / nc;
  lo = (size_t)c * per;
  hi = lo + per;
  if (hi > len) hi = len;
  if (lo > len) lo = len;
}

// stage 1 of dot / norm: partial[(rhs * ndots + d) * nc + chunk] (re, im)
template <typename T>
__global__ void k_multidot1(double* __restrict__ part, const cplx<T>* __restrict__ V, size_t vstride, int m,
                            const cplx<T>* __restrict__ w, size_t len, size_t rstride, int nc) {
  __shared__ double sh[32 * 8];
  const int chunk = blockIdx.x, rhs = blockIdx.y;
  size_t lo, hi;
  chunk_range(len, nc, chunk, lo, hi);
  const cplx<T>* pw = w + (size_t)rhs * rstride;
  for (int d0 = 0; d0 < m; d0 += 4) {
    // per-thread partials in the precision of the data (FP32 data: FP32 sums)
    T at[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (size_t e = lo + threadIdx.x; e < hi; e += blockDim.x) {
      const cplx<T> we = pw[e];
#pragma unroll
      for (int dd = 0; dd < 4; ++dd) {
        if (d0 + dd < m) {
          const cplx<T> v = V[(size_t)(d0 + dd) * vstride + (size_t)rhs * rstride + e];
          cdotc_acc(at[2 * dd], at[2 * dd + 1], v, we);
        }
      }
    }
    double acc[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = (double)at[k];
    cta_sum(acc, 8, sh);
    if (threadIdx.x == 0)
      for (int dd = 0; dd < 4 && d0 + dd < m; ++dd) {
        double* p = part + (((size_t)rhs * m + d0 + dd) * nc + chunk) * 2;
        p[0] = acc[2 * dd];
        p[1] = acc[2 * dd + 1];
      }
  }
}

// stage 1 of the multidot in double-FP32 arithmetic on FP64 vectors: the elements are split on
// load, products and the per-thread sums are double-FP32, the CTA sum is FP64 (partials as above)
__global__ void k_multidot1_df(double* __restrict__ part, const cplx<double>* __restrict__ V, size_t vstride,
                               int m, const cplx<double>* __restrict__ w, size_t len, size_t rstride, int nc) {
  __shared__ double sh[32 * 8];
  const int chunk = blockIdx.x, rhs = blockIdx.y;
  size_t lo, hi;
  chunk_range(len, nc, chunk, lo, hi);
  const cplx<double>* pw = w + (size_t)rhs * rstride;
  for (int d0 = 0; d0 < m; d0 += 4) {
    dfl at[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) at[k] = dfl(0);
    for (size_t e = lo + threadIdx.x; e < hi; e += blockDim.x) {
      const cplx<double> wd = pw[e];
      const dfl wr = df_from_double(wd.re), wi = df_from_double(wd.im);
#pragma unroll
      for (int dd = 0; dd < 4; ++dd) {
        if (d0 + dd < m) {
          const cplx<double> vd = V[(size_t)(d0 + dd) * vstride + (size_t)rhs * rstride + e];
          const dfl vr = df_from_double(vd.re), vi = df_from_double(vd.im);
          // conj(v) w
          at[2 * dd] = fma(vr, wr, at[2 * dd]);
          at[2 * dd] = fma(vi, wi, at[2 * dd]);
          at[2 * dd + 1] = fma(vr, wi, at[2 * dd + 1]);
          at[2 * dd + 1] = fma(-vi, wr, at[2 * dd + 1]);
        }
      }
    }
    double acc[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = df_to_double(at[k]);
    cta_sum(acc, 8, sh);
    if (threadIdx.x == 0)
      for (int dd = 0; dd < 4 && d0 + dd < m; ++dd) {
        double* p = part + (((size_t)rhs * m + d0 + dd) * nc + chunk) * 2;
        p[0] = acc[2 * dd];
        p[1] = acc[2 * dd + 1];
      }
  }
}

// stage 2: res[rhs * m + d] = sum over chunks, fixed order
__global__ void k_multidot2(cplx<double>* __restrict__ res, const double* __restrict__ part, int m, int nc,
                            int res_stride) {
  __shared__ double sh[32 * 8];
  const int d = blockIdx.x, rhs = blockIdx.y;
  const double* p = part + ((size_t)rhs * m + d) * nc * 2;
  double acc[2] = {0.0, 0.0};
  for (int c = threadIdx.x; c < nc; c += blockDim.x) { acc[0] += p[2 * c]; acc[1] += p[2 * c + 1]; }
  cta_sum(acc, 2, sh);
  if (threadIdx.x == 0) res[(size_t)rhs * res_stride + d] = cmk(acc[0], acc[1]);
}

template <typename T>
__global__ void k_norm1(double* __restrict__ part, const cplx<T>* __restrict__ x, size_t len, size_t rstride, int nc) {
  __shared__ double sh[32 * 8];
  const int chunk = blockIdx.x, rhs = blockIdx.y;
  size_t lo, hi;
  chunk_range(len, nc, chunk, lo, hi);
  const cplx<T>* px = x + (size_t)rhs * rstride;
  T at = T(0);
  for (size_t e = lo + threadIdx.x; e < hi; e += blockDim.x) {
    const cplx<T> v = px[e];
    cnorm2_acc(at, v);
  }
  double acc[1] = {(double)at};
  cta_sum(acc, 1, sh);
  if (threadIdx.x == 0) part[(size_t)rhs * nc + chunk] = acc[0];
}

__global__ void k_norm2(double* __restrict__ res, const double* __restrict__ part, int nc) {
  __shared__ double sh[32 * 8];
  const int rhs = blockIdx.x;
  double acc[1] = {0.0};
  for (int c = threadIdx.x; c < nc; c += blockDim.x) acc[0] += part[(size_t)rhs * nc + c];
  cta_sum(acc, 1, sh);
  if (threadIdx.x == 0) res[rhs] = sqrt(acc[0]);
}

template <typename T>
__global__ void k_multiaxpy(cplx<T>* __restrict__ y, const cplx<T>* __restrict__ V, size_t vstride, int m,
                            const cplx<double>* __restrict__ c, int cstride, double sign, size_t len,
                            size_t rstride) {
  // coefficients sign * c_i of this right-hand side, computed once per CTA; a zero
  // coefficient skips its vector (never touch unused, possibly unset vectors)
  __shared__ cplx<T> cs[64];
  __shared__ int use[64];
  const int rhs = blockIdx.y;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const cplx<double> ci = c[(size_t)rhs * cstride + i];
    use[i] = !(ci.re == 0.0 && ci.im == 0.0);
    cs[i] = cmk<T>((T)(sign * ci.re), (T)(sign * ci.im));
  }
  __syncthreads();
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= len) return;
  const size_t o = (size_t)rhs * rstride + e;
  cplx<T> acc = y[o];
  for (int i = 0; i < m; ++i) {
    if (!use[i]) continue;
    cfma(acc, cs[i], V[(size_t)i * vstride + o]);
  }
  y[o] = acc;
}

// y += sign * sum_i c_i V_i in double-FP32 arithmetic on FP64 vectors (result rounded to FP64)
__global__ void k_multiaxpy_df(cplx<double>* __restrict__ y, const cplx<double>* __restrict__ V, size_t vstride,
                               int m, const cplx<double>* __restrict__ c, int cstride, double sign, size_t len,
                               size_t rstride) {
  __shared__ cplx<dfl> cs[64];
  __shared__ int use[64];
  const int rhs = blockIdx.y;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const cplx<double> ci = c[(size_t)rhs * cstride + i];
    use[i] = !(ci.re == 0.0 && ci.im == 0.0);
    const double a = sign * ci.re, b = sign * ci.im;
    const float ah = __double2float_rn(a), bh = __double2float_rn(b);
    cs[i] = cmk<dfl>(dfl(ah, __double2float_rn(a - (double)ah)), dfl(bh, __double2float_rn(b - (double)bh)));
  }
  __syncthreads();
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= len) return;
  const size_t o = (size_t)rhs * rstride + e;
  const cplx<double> yd = y[o];
  cplx<dfl> acc = cmk<dfl>(df_from_double(yd.re), df_from_double(yd.im));
  for (int i = 0; i < m; ++i) {
    if (!use[i]) continue;
    const cplx<double> vd = V[(size_t)i * vstride + o];
    cfma(acc, cs[i], cmk<dfl>(df_from_double(vd.re), df_from_double(vd.im)));
  }
  y[o] = cmk<double>(df_to_double(acc.re), df_to_double(acc.im));
}

template <typename T>
__global__ void k_scale_to(cplx<T>* y, const cplx<T>* x, const double* __restrict__ a,
                           size_t len, size_t rstride) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= len) return;
  const size_t o = (size_t)blockIdx.y * rstride + e;
  const T s = (T)a[blockIdx.y];
  y[o] = s * x[o];
}

template <typename T>
__global__ void k_axpy(cplx<T>* __restrict__ y, const cplx<T>* __restrict__ x, double a, size_t len, size_t rstride) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= len) return;
  const size_t o = (size_t)blockIdx.y * rstride + e;
  y[o] = y[o] + (T)a * x[o];
}

template <typename To, typename Ti>
__global__ void k_convert(cplx<To>* y, const cplx<Ti>* x, size_t len, size_t ys, size_t xs) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= len) return;
  y[(size_t)blockIdx.y * ys + e] = ccast<To>(x[(size_t)blockIdx.y * xs + e]);
}

template <typename T>
__global__ void k_zero(cplx<T>* __restrict__ y, size_t len, size_t rstride) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= len) return;
  y[(size_t)blockIdx.y * rstride + e] = czero<T>();
}

__global__ void k_recip(double* __restrict__ a, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = a[i] > 0.0 ? 1.0 / a[i] : 0.0;
}

template <typename T>
__global__ void k_real_convert(T* __restrict__ y, const double* __restrict__ x, size_t len) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < len) y[e] = (T)x[e];
}

// ---- GMRES (one thread per rhs) ----------------------------------------------
// Givens convention: [[c, s], [-conj(s), c]] (a, b)^T = (rho, 0)^T with c real.
__device__ void givens(cplx<double> a, cplx<double> b, double& c, cplx<double>& s) {
  const double aa = sqrt(cnorm2(a)), bb = sqrt(cnorm2(b));
  const double r = hypot(aa, bb);
  if (r == 0.0) { c = 1.0; s = czero<double>(); return; }
  if (aa == 0.0) { c = 0.0; s = bb == 0.0 ? cmk(1.0, 0.0) : cmk(b.re / bb, -b.im / bb); return; }
  c = aa / r;
  const cplx<double> ph = cmk(a.re / aa, a.im / aa);
  s = (1.0 / r) * (ph * cconj(b));
}

__global__ void k_gmres_begin(dd::GmresState s, int nrhs) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs) return;
  const int m = s.m;
  for (int k = 0; k <= m; ++k) s.g[(size_t)r * (m + 1) + k] = czero<double>();
  const double b = s.beta[r];
  s.g[(size_t)r * (m + 1)] = cmk(b, 0.0);
  s.kr[r] = 0;
  s.done[r] = (b <= s.target[r]) ? 1 : 0;
  s.inv[r] = (b > 0.0 && !s.done[r]) ? 1.0 / b : 0.0;
  s.est[r] = b;
}

__global__ void k_gmres_step(dd::GmresState s, int j, int nrhs) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs) return;
  if (s.done[r]) { s.inv[r] = 0.0; return; }   // finished rhs: next basis vector is exactly zero
  const int m = s.m;
  cplx<double>* H = s.H + (size_t)r * (m + 1) * m;
  cplx<double>* g = s.g + (size_t)r * (m + 1);
  double* cs = s.cs + (size_t)r * m;
  cplx<double>* sn = s.sn + (size_t)r * m;
  cplx<double> h[64];
  for (int i = 0; i <= j; ++i) h[i] = s.h1[(size_t)r * (m + 1) + i] + s.h2[(size_t)r * (m + 1) + i];
  const double hn = s.wnorm[r];
  h[j + 1] = cmk(hn, 0.0);
  for (int i = 0; i < j; ++i) {
    const cplx<double> t = cs[i] * h[i] + sn[i] * h[i + 1];
    h[i + 1] = cs[i] * h[i + 1] - cconj(sn[i]) * h[i];
    h[i] = t;
  }
  double c;
  cplx<double> sg;
  givens(h[j], h[j + 1], c, sg);
  cs[j] = c;
  sn[j] = sg;
  h[j] = c * h[j] + sg * h[j + 1];
  h[j + 1] = czero<double>();
  g[j + 1] = -1.0 * (cconj(sg) * g[j]);
  g[j] = c * g[j];
  for (int i = 0; i <= j + 1; ++i) H[(size_t)i * m + j] = h[i];
  s.kr[r] = j + 1;
  const double est = sqrt(cnorm2(g[j + 1]));
  s.est[r] = est;
  s.inv[r] = hn > 0.0 ? 1.0 / hn : 0.0;
  if (est <= s.target[r] || hn == 0.0 || j + 1 == m) { s.done[r] = 1; s.inv[r] = 0.0; }
}

__global__ void k_gmres_solve_y(dd::GmresState s, int nrhs) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs) return;
  const int m = s.m;
  const int k = s.kr[r];
  const cplx<double>* H = s.H + (size_t)r * (m + 1) * m;
  const cplx<double>* g = s.g + (size_t)r * (m + 1);
  cplx<double>* y = s.y + (size_t)r * m;
  for (int i = k; i < m; ++i) y[i] = czero<double>();
  for (int i = k - 1; i >= 0; --i) {
    cplx<double> t = g[i];
    for (int l = i + 1; l < k; ++l) t = t - H[(size_t)i * m + l] * y[l];
    const cplx<double> d = H[(size_t)i * m + i];
    const double dn = cnorm2(d);
    y[i] = dn > 0.0 ? (1.0 / dn) * (t * cconj(d)) : czero<double>();
  }
}

}  // namespace

namespace dd {

static std::atomic<long long> g_launches{0};
void count_launch(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

template <typename T>
void blas_multidot(cplx<double>* res, int res_stride, const cplx<T>* V, size_t vstride, int m, const cplx<T>* w,
                   size_t len, int nrhs, size_t rstride, cudaStream_t st) {
  if (m <= 0) return;
  const int nc = nchunks(len);
  double* part = partials((size_t)nrhs * m * nc * 2, st);
  count_launch();
  k_multidot1<T><<<dim3(nc, nrhs), RT, 0, st>>>(part, V, vstride, m, w, len, rstride, nc);
  count_launch();
  k_multidot2<<<dim3(m, nrhs), 128, 0, st>>>(res, part, m, nc, res_stride);
}

void blas_multidot_df(cplx<double>* res, int res_stride, const cplx<double>* V, size_t vstride, int m,
                      const cplx<double>* w, size_t len, int nrhs, size_t rstride, cudaStream_t st) {
  if (m <= 0) return;
  const int nc = nchunks(len);
  double* part = partials((size_t)nrhs * m * nc * 2, st);
  count_launch();
  k_multidot1_df<<<dim3(nc, nrhs), RT, 0, st>>>(part, V, vstride, m, w, len, rstride, nc);
  count_launch();
  k_multidot2<<<dim3(m, nrhs), 128, 0, st>>>(res, part, m, nc, res_stride);
}

void blas_multiaxpy_df(cplx<double>* y, const cplx<double>* V, size_t vstride, int m, const cplx<double>* c,
                       int cstride, double sign, size_t len, int nrhs, size_t rstride, cudaStream_t st) {
  if (m <= 0) return;
  if (m > 64) throw std::runtime_error("blas_multiaxpy_df: at most 64 vectors");
  count_launch();
  k_multiaxpy_df<<<dim3(div_up(len, 256), nrhs), 256, 0, st>>>(y, V, vstride, m, c, cstride, sign, len, rstride);
}

void reserve_partials(int nrhs, int m, cudaStream_t st) { partials((size_t)nrhs * (m + 1) * MAXCHUNKS * 2, st); }

template <typename T>
void blas_dot(cplx<double>* res, const cplx<T>* x, const cplx<T>* y, size_t len, int nrhs, size_t rstride,
              cudaStream_t st) {
  blas_multidot<T>(res, 1, x, 0, 1, y, len, nrhs, rstride, st);
}

template <typename T>
void blas_norm2(double* res, const cplx<T>* x, size_t len, int nrhs, size_t rstride, cudaStream_t st) {
  const int nc = nchunks(len);
  double* part = partials((size_t)nrhs * nc, st);
  count_launch();
  k_norm1<T><<<dim3(nc, nrhs), RT, 0, st>>>(part, x, len, rstride, nc);
  count_launch();
  k_norm2<<<nrhs, 128, 0, st>>>(res, part, nc);
}

template <typename T>
void blas_multiaxpy(cplx<T>* y, const cplx<T>* V, size_t vstride, int m, const cplx<double>* c, int cstride,
                    double sign, size_t len, int nrhs, size_t rstride, cudaStream_t st) {
  if (m <= 0) return;
  if (m > 64) throw std::runtime_error("blas_multiaxpy: at most 64 vectors");
  count_launch();
  k_multiaxpy<T><<<dim3(div_up(len, 256), nrhs), 256, 0, st>>>(y, V, vstride, m, c, cstride, sign, len, rstride);
}

template <typename T>
void blas_scale_to(cplx<T>* y, const cplx<T>* x, const double* a, size_t len, int nrhs, size_t rstride,
                   cudaStream_t st) {
  count_launch();
  k_scale_to<T><<<dim3(div_up(len, 256), nrhs), 256, 0, st>>>(y, x, a, len, rstride);
}

template <typename T>
void blas_axpy(cplx<T>* y, const cplx<T>* x, double a, size_t len, int nrhs, size_t rstride, cudaStream_t st) {
  count_launch();
  k_axpy<T><<<dim3(div_up(len, 256), nrhs), 256, 0, st>>>(y, x, a, len, rstride);
}

template <typename To, typename Ti>
void blas_convert(cplx<To>* y, const cplx<Ti>* x, size_t len, int nrhs, size_t ystride, size_t xstride,
                  cudaStream_t st) {
  count_launch();
  k_convert<To, Ti><<<dim3(div_up(len, 256), nrhs), 256, 0, st>>>(y, x, len, ystride, xstride);
}

template <typename T>
void blas_zero(cplx<T>* y, size_t len, int nrhs, size_t rstride, cudaStream_t st) {
  count_launch();
  k_zero<T><<<dim3(div_up(len, 256), nrhs), 256, 0, st>>>(y, len, rstride);
}

template <typename T>
void real_convert(T* y, const double* x, size_t len, cudaStream_t st) {
  count_launch();
  k_real_convert<T><<<div_up(len, 256), 256, 0, st>>>(y, x, len);
}

void blas_recip(double* a, int n, cudaStream_t st) { k_recip<<<div_up(n, 128), 128, 0, st>>>(a, n); }

void gmres_begin(const GmresState& s, int nrhs, cudaStream_t st) { k_gmres_begin<<<div_up(nrhs, 32), 32, 0, st>>>(s, nrhs); }
void gmres_step(const GmresState& s, int j, int nrhs, cudaStream_t st) {
  count_launch();
  k_gmres_step<<<div_up(nrhs, 32), 32, 0, st>>>(s, j, nrhs);
}
void gmres_solve_y(const GmresState& s, int nrhs, cudaStream_t st) {
  count_launch();
  k_gmres_solve_y<<<div_up(nrhs, 32), 32, 0, st>>>(s, nrhs);
}

#define INST(T)                                                                                                 \
  template void blas_multidot<T>(cplx<double>*, int, const cplx<T>*, size_t, int, const cplx<T>*, size_t, int,   \
                                 size_t, cudaStream_t);                                                         \
  template void blas_dot<T>(cplx<double>*, const cplx<T>*, const cplx<T>*, size_t, int, size_t, cudaStream_t);   \
  template void blas_norm2<T>(double*, const cplx<T>*, size_t, int, size_t, cudaStream_t);                      \
  template void blas_multiaxpy<T>(cplx<T>*, const cplx<T>*, size_t, int, const cplx<double>*, int, double,      \
                                  size_t, int, size_t, cudaStream_t);                                           \
  template void blas_scale_to<T>(cplx<T>*, const cplx<T>*, const double*, size_t, int, size_t, cudaStream_t);   \
  template void blas_axpy<T>(cplx<T>*, const cplx<T>*, double, size_t, int, size_t, cudaStream_t);              \
  template void blas_zero<T>(cplx<T>*, size_t, int, size_t, cudaStream_t);                                      \
  template void real_convert<T>(T*, const double*, size_t, cudaStream_t);
INST(float)
INST(double)
#undef INST
template void blas_convert<float, double>(cplx<float>*, const cplx<double>*, size_t, int, size_t, size_t, cudaStream_t);
template void blas_convert<double, float>(cplx<double>*, const cplx<float>*, size_t, int, size_t, size_t, cudaStream_t);
template void blas_convert<double, double>(cplx<double>*, const cplx<double>*, size_t, int, size_t, size_t,
                                           cudaStream_t);
template void blas_convert<float, float>(cplx<float>*, const cplx<float>*, size_t, int, size_t, size_t, cudaStream_t);

}  // namespace dd
