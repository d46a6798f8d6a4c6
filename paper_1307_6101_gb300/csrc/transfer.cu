// Aggregation-based transfer operators (Sec. 1, Sec. 2.2 of the paper).
//
// P_l is stored as the N orthonormalised test-vector fields of level l.  For
// aggregate A and chirality s (spins 0,1 / 2,3 on the fine level, first and
// second half of the dof on a coarse level), column j of the block
// Q_{A,s} is field j restricted to (A, s); coarse dof (A, s, j) has index s*N + j.
// Aggregates are contiguous index ranges [A*vA, (A+1)*vA) in the site order.
#include "common.cuh"
#include "kernels.h"

namespace {

// address of (site x, component f) in a level field: fine [12][V], coarse [V][n]
DD_HD size_t faddr(bool fine, int V, int n, int x, int f) {
  return fine ? (size_t)f * V + x : (size_t)x * n + f;
}


template <typename T>
__device__ void block_sum(T* v, int cnt, T* sh) {
  // sum cnt values per thread over the CTA; result valid in every thread
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int k = 0; k < cnt; ++k)
    for (int off = 16; off >= 1; off >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], off);
  if (lane == 0)
    for (int k = 0; k < cnt; ++k) sh[warp * cnt + k] = v[k];
  __syncthreads();
  for (int k = 0; k < cnt; ++k) {
    T s = T(0);
    for (int w = 0; w < nw; ++w) s += sh[w * cnt + k];
    v[k] = s;
  }
  __syncthreads();
}

constexpr int RJ = 10;   // coarse columns j accumulated per thread by k_restrict

// out(A)[s*N + j] = sum over x in A, f in s of conj(P_j(x, f)) in(x, f).
// One CTA per aggregate (and right-hand side); thread (group g, lane l) owns the
// columns j in [g*RJ, g*RJ + RJ) and the sites x = A*vA + l, l + S, ... of the
// aggregate, so every input and every P entry is loaded once.  S is a power of
// two; the per-thread partial sums are reduced over the S lanes of a group in a
// fixed order (shuffles inside warps, then shared memory across warps).  HF > 0:
// the fine level, whose HF = 6 dofs per chirality are unrolled so that all loads
// of a chirality are in flight together.
template <typename T, typename PS, int HF>
__global__ void __launch_bounds__(512, HF > 0 ? 1 : 2) k_restrict(cplx<T>* __restrict__ out, const cplx<T>* __restrict__ in, const PS* __restrict__ P,
                           const float* __restrict__ pscale, Geom gf, Geom gc, bool fine, int n, int N, int S,
                           size_t in_rstride, size_t pstride, size_t out_rstride, size_t out_site_stride) {
  __shared__ T red[32 * 2 * RJ];
  const int agg = blockIdx.x;
  const int V = gf.V;
  const cplx<T>* pin = in + (size_t)blockIdx.y * in_rstride;
  int c0[4];
  geom_coords(gf, agg * gf.vA, c0);   // first site of the aggregate (aggregates are contiguous)
  const int cs = coarse_site_of(gf, gc, c0);
  cplx<T>* po = out + (size_t)blockIdx.y * out_rstride + (size_t)cs * out_site_stride;
  const int h = n / 2;
  const int seg = S < 32 ? S : 32;            // lanes of a group inside one warp
  const int slots = S / seg;                  // partial sums per group after the warp stage
  const int gpc = blockDim.x / S;             // groups per CTA
  const int G = (N + RJ - 1) / RJ;            // column groups
  const int lane = threadIdx.x % S;
  for (int g0 = 0; g0 < G; g0 += gpc) {
    const int g = g0 + threadIdx.x / S;
    const int j0 = g * RJ;
    for (int s = 0; s < 2; ++s) {
      T acc[2 * RJ];
#pragma unroll
      for (int k = 0; k < 2 * RJ; ++k) acc[k] = T(0);
      if (g < G) {
        for (int xl = lane; xl < gf.vA; xl += S) {
          const int x = agg * gf.vA + xl;
          if constexpr (HF > 0) {
            cplx<T> v[HF];
#pragma unroll
            for (int f = 0; f < HF; ++f) v[f] = pin[(size_t)(s * HF + f) * V + x];
#pragma unroll
            for (int jj = 0; jj < RJ; ++jj)
              if (j0 + jj < N)
#pragma unroll
                for (int f = 0; f < HF; ++f)
                  cdotc_acc(acc[2 * jj], acc[2 * jj + 1],
                            ld_cplx(P, (size_t)(j0 + jj) * pstride + (size_t)(s * HF + f) * V + x), v[f]);
          } else {
            for (int f = s * h; f < (s + 1) * h; ++f) {
              const size_t a = faddr(fine, V, n, x, f);
              const cplx<T> v = pin[a];
#pragma unroll
              for (int jj = 0; jj < RJ; ++jj)
                if (j0 + jj < N) cdotc_acc(acc[2 * jj], acc[2 * jj + 1], ld_cplx(P, (size_t)(j0 + jj) * pstride + a), v);
            }
          }
        }
      }
      for (int off = seg / 2; off >= 1; off >>= 1)
#pragma unroll
        for (int k = 0; k < 2 * RJ; ++k) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], off);
      if (threadIdx.x % seg == 0)
#pragma unroll
        for (int k = 0; k < 2 * RJ; ++k) red[(threadIdx.x / seg) * 2 * RJ + k] = acc[k];
      __syncthreads();
      for (int t = threadIdx.x; t < gpc * RJ; t += blockDim.x) {
        const int gl = t / RJ, jj = t % RJ;
        const int j = (g0 + gl) * RJ + jj;
        if (g0 + gl < G && j < N) {
          T re = T(0), im = T(0);
          for (int q = 0; q < slots; ++q) {
            re += red[(gl * slots + q) * 2 * RJ + 2 * jj];
            im += red[(gl * slots + q) * 2 * RJ + 2 * jj + 1];
          }
          const T sc = pscale ? T(pscale[agg * 2 + s]) : T(1);
          po[s * N + j] = cmk<T>(sc * re, sc * im);
        }
      }
      __syncthreads();
    }
  }
}

template <typename T, typename PS>
__global__ void k_prolong(cplx<T>* __restrict__ out, const cplx<T>* __restrict__ in, const PS* __restrict__ P,
                          const float* __restrict__ pscale, Geom gf, Geom gc, bool fine, int n, int N,
                          size_t out_rstride, size_t in_rstride, size_t pstride, bool accumulate) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int V = gf.V;
  if (t >= (size_t)V * n) return;
  int x, f;
  if (fine) { f = (int)(t / V); x = (int)(t % V); }
  else { x = (int)(t / n); f = (int)(t % n); }
  int c[4];
  geom_coords(gf, x, c);
  const int cs = coarse_site_of(gf, gc, c);
  const int s = f < n / 2 ? 0 : 1;
  const cplx<T>* pc = in + (size_t)blockIdx.y * in_rstride + (size_t)cs * (2 * N) + s * N;
  cplx<T> acc = czero<T>();
  const size_t a = faddr(fine, V, n, x, f);
  for (int j = 0; j < N; ++j) cfma(acc, ld_cplx(P, (size_t)j * pstride + a), pc[j]);
  if (pscale) acc = T(pscale[(x / gf.vA) * 2 + s]) * acc;
  cplx<T>* po = out + (size_t)blockIdx.y * out_rstride + a;
  *po = accumulate ? *po + acc : acc;
}

// CGS2 of the N test vectors restricted to (aggregate, chirality), in column order.
__global__ void k_orthonormalise(cplx<double>* __restrict__ P, Geom g, bool fine, int n, int N, size_t pstride,
                                 int* err) {
  __shared__ double sh[32 * 2 * 8];
  __shared__ cplx<double> hs[64];
  const int agg = blockIdx.x;
  const int s = blockIdx.y;
  const int h = n / 2;
  const int ne = g.vA * h;
  const int V = g.V;
  auto addr = [&](int e) {
    const int x = agg * g.vA + e / h;
    const int f = s * h + e % h;
    return faddr(fine, V, n, x, f);
  };
  for (int j = 0; j < N; ++j) {
    cplx<double>* w = P + (size_t)j * pstride;
    double n0 = 0.0;
    for (int e = threadIdx.x; e < ne; e += blockDim.x) n0 += cnorm2(w[addr(e)]);
    block_sum(&n0, 1, sh);
    for (int pass = 0; pass < 2; ++pass) {
      for (int i0 = 0; i0 < j; i0 += 8) {
        double acc[16];
        for (int k = 0; k < 16; ++k) acc[k] = 0.0;
        for (int e = threadIdx.x; e < ne; e += blockDim.x) {
          const size_t a = addr(e);
          const cplx<double> we = w[a];
          for (int ii = 0; ii < 8 && i0 + ii < j; ++ii) {
            const cplx<double> t = cdotc(P[(size_t)(i0 + ii) * pstride + a], we);
            acc[2 * ii] += t.re;
            acc[2 * ii + 1] += t.im;
          }
        }
        block_sum(acc, 16, sh);
        if (threadIdx.x < 8 && i0 + threadIdx.x < j) hs[i0 + threadIdx.x] = cmk(acc[2 * threadIdx.x], acc[2 * threadIdx.x + 1]);
      }
      __syncthreads();
      for (int e = threadIdx.x; e < ne; e += blockDim.x) {
        const size_t a = addr(e);
        cplx<double> we = w[a];
        for (int i = 0; i < j; ++i) we = we - hs[i] * P[(size_t)i * pstride + a];
        w[a] = we;
      }
      __syncthreads();
    }
    double nn = 0.0;
    for (int e = threadIdx.x; e < ne; e += blockDim.x) nn += cnorm2(w[addr(e)]);
    block_sum(&nn, 1, sh);
    const double nrm = sqrt(nn);
    if (!(nrm > 1e-12 * sqrt(n0)) || n0 == 0.0) {
      if (threadIdx.x == 0) atomicExch(err, 1);
      return;
    }
    const double inv = 1.0 / nrm;
    for (int e = threadIdx.x; e < ne; e += blockDim.x) {
      const size_t a = addr(e);
      w[a] = inv * w[a];
    }
    __syncthreads();
  }
}

// FP16 copy of P with one scale per (aggregate, chirality): s = float(max |re|, |im|)
// over the N columns restricted to (A, s), q = RNE_half(x / s).
__global__ void k_p_to_half(__half2* __restrict__ Ph, float* __restrict__ pscale, const cplx<double>* __restrict__ P,
                            Geom g, bool fine, int n, int N, size_t pstride) {
  __shared__ double sh[32];
  const int agg = blockIdx.x, s = blockIdx.y, h = n / 2;
  const int ne = g.vA * h;
  const int V = g.V;
  double mx = 0.0;
  for (int j = 0; j < N; ++j)
    for (int e = threadIdx.x; e < ne; e += blockDim.x) {
      const cplx<double> v = P[(size_t)j * pstride + faddr(fine, V, n, agg * g.vA + e / h, s * h + e % h)];
      mx = fmax(mx, fmax(fabs(v.re), fabs(v.im)));
    }
  for (int off = 16; off >= 1; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, sh[w]);
    const float sf = m > 0.0 ? (float)m : 1.0f;
    pscale[agg * 2 + s] = sf;
    sh[0] = (double)sf;
  }
  __syncthreads();
  const double sc = sh[0];
  for (int j = 0; j < N; ++j)
    for (int e = threadIdx.x; e < ne; e += blockDim.x) {
      const size_t a = (size_t)j * pstride + faddr(fine, V, n, agg * g.vA + e / h, s * h + e % h);
      Ph[a] = __halves2half2(__double2half(P[a].re / sc), __double2half(P[a].im / sc));
    }
}

}  // namespace

namespace dd {

void p_to_half(__half2* Ph, float* pscale, const cplx<double>* P, const Geom& g, bool fine, int n, int N,
               cudaStream_t st) {
  count_launch();
  k_p_to_half<<<dim3(g.nAgg, 2), 256, 0, st>>>(Ph, pscale, P, g, fine, n, N, (size_t)g.V * n);
}

template <typename T>
void restrict_op(cplx<T>* out, const cplx<T>* in, const cplx<T>* P, const Geom& gf, const Geom& gc, bool fine, int n,
                 int N, int nrhs, size_t in_rstride, size_t out_rstride, size_t out_site_stride, cudaStream_t st,
                 const __half2* Ph, const float* pscale, int tc_ks) {
  if constexpr (sizeof(T) == 4) {
    // FP16 P: the tensor-core kernel (P read once per batch) where the autotuner chose it
    if (Ph && tc_ks > 0) {
      if (restrict_tc(out, in, Ph, pscale, gf, gc, fine, n, N, nrhs, in_rstride, out_rstride, out_site_stride, tc_ks,
                      st) == cudaSuccess)
        return;
      cudaGetLastError();
    }
  }
  const size_t pstride = (size_t)gf.V * n;
  int S = 1;   // lanes per column group: a power of two >= the aggregate volume, at most 256
  while (S < gf.vA && S < 256) S *= 2;
  const int G = (N + RJ - 1) / RJ;
  int gpc = 512 / S < G ? 512 / S : G;   // at most 512 threads (launch bounds)
  if (S < 32) gpc = ((gpc * S + 31) / 32) * (32 / S);   // whole warps (the shuffles use full masks)
  if (S < 32 && gpc > 32) gpc = 32;                     // partial-sum slots in shared memory
  const int threads = gpc * S;
  count_launch();
  const dim3 grid(gf.nAgg, nrhs);
  if constexpr (sizeof(T) == 4) {
    if (Ph) {
      if (fine)
        k_restrict<float, __half2, 6><<<grid, threads, 0, st>>>(out, in, Ph, pscale, gf, gc, fine, n, N, S, in_rstride,
                                                                 pstride, out_rstride, out_site_stride);
      else
        k_restrict<float, __half2, 0><<<grid, threads, 0, st>>>(out, in, Ph, pscale, gf, gc, fine, n, N, S, in_rstride,
                                                                 pstride, out_rstride, out_site_stride);
      return;
    }
  }
  if (fine)
    k_restrict<T, cplx<T>, 6><<<grid, threads, 0, st>>>(out, in, P, nullptr, gf, gc, fine, n, N, S, in_rstride,
                                                          pstride, out_rstride, out_site_stride);
  else
    k_restrict<T, cplx<T>, 0><<<grid, threads, 0, st>>>(out, in, P, nullptr, gf, gc, fine, n, N, S, in_rstride,
                                                          pstride, out_rstride, out_site_stride);
}

template <typename T>
void prolong_op(cplx<T>* out, const cplx<T>* in, const cplx<T>* P, const Geom& gf, const Geom& gc, bool fine, int n,
                int N, int nrhs, size_t out_rstride, size_t in_rstride, bool accumulate, cudaStream_t st,
                const __half2* Ph, const float* pscale, int batch) {
  if constexpr (sizeof(T) == 4) {
    // FP16 P: one CTA per aggregate for the whole batch (P read once) where the autotuner chose it
    if (Ph && batch) {
      if (prolong_batch(out, in, Ph, pscale, gf, gc, fine, n, N, nrhs, out_rstride, in_rstride, accumulate, st) ==
          cudaSuccess)
        return;
      cudaGetLastError();
    }
  }
  const size_t pstride = (size_t)gf.V * n;
  const size_t tot = (size_t)gf.V * n;
  count_launch();
  if constexpr (sizeof(T) == 4) {
    if (Ph) {
      k_prolong<float, __half2><<<dim3(div_up(tot, 128), nrhs), 128, 0, st>>>(
          out, in, Ph, pscale, gf, gc, fine, n, N, out_rstride, in_rstride, pstride, accumulate);
      return;
    }
  }
  k_prolong<T, cplx<T>><<<dim3(div_up(tot, 128), nrhs), 128, 0, st>>>(out, in, P, nullptr, gf, gc, fine, n, N,
                                                                       out_rstride, in_rstride, pstride, accumulate);
}

void orthonormalise(cplx<double>* P, const Geom& g, bool fine, int n, int N, int* err, cudaStream_t st) {
  const size_t pstride = (size_t)g.V * n;
  count_launch();
  k_orthonormalise<<<dim3(g.nAgg, 2), 256, 0, st>>>(P, g, fine, n, N, pstride, err);
}

#define INST(T)                                                                                                  \
  template void restrict_op<T>(cplx<T>*, const cplx<T>*, const cplx<T>*, const Geom&, const Geom&, bool, int, int, \
                               int, size_t, size_t, size_t, cudaStream_t, const __half2*, const float*, int);   \
  template void prolong_op<T>(cplx<T>*, const cplx<T>*, const cplx<T>*, const Geom&, const Geom&, bool, int, int,  \
                              int, size_t, size_t, bool, cudaStream_t, const __half2*, const float*, int);
INST(float)
INST(double)
#undef INST

}  // namespace dd
