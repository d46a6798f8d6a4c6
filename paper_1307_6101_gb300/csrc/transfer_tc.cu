// Transfer operators for a batch of right-hand sides, reading P once per batch (Sec. 1: the
// restriction P^dagger and the interpolation P built from the aggregated test vectors, Sec. 2.2).
//
// Restriction on tensor cores: for aggregate A and chirality s,
//   out(A)[s N + j][r] = sum_{x in A, f in s} conj(P_j(x, f)) in_r(x, f),
// an (N x K) by (K x R) product with K = |A| * n/2, done in chunks of K; per chunk the FP16 P entries
// (exact operands; the per-(A, s) FP32 scale multiplies the result) and each right-hand side's
// values, scaled by a power of two s_r >= their max |Re|, |Im| in the chunk and split into FP16
// hi + lo parts, are staged in shared memory and multiplied by mma.sync m16n8k16 (FP32 accumulate)
// in the real form  [Re y; Im y] = [[Re p, Im p], [-Im p, Re p]] [Re x; Im x];  chunk results are
// added as s_r * partial in a fixed order.  A column's result depends only on that column.
//
// Interpolation on CUDA cores: one CTA per aggregate stages the aggregate's coarse values of every
// right-hand side in shared memory; a thread owns one (site, component) row, loads its N entries of
// P once and forms the row for every right-hand side of the batch (same order for every column).
#include "common.cuh"
#include "kernels.h"

#include <atomic>
#include <mutex>

namespace {

constexpr int RT_R = 16;     // right-hand sides per CTA of the restriction
constexpr int RT_KCH = 192;  // complex K entries per chunk (24 k-tiles of 8)
constexpr int RT_PS = RT_KCH + 8;   // row stride (words) of the staged P chunk: = 8 mod 32
constexpr int RT_XS = RT_KCH + 4;   // row stride (8-byte slots) of the staged vectors: = 4 mod 16

__device__ __forceinline__ void mma_16816(float c[4], const unsigned a[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

DD_HD size_t faddr(bool fine, int V, int n, int x, int f) { return fine ? (size_t)f * V + x : (size_t)x * n + f; }

__host__ __device__ inline size_t rt_smem(int N, int ks) {
  const int mt = (2 * N + 15) / 16;
  return (size_t)N * RT_PS * 4 + (size_t)RT_R * RT_XS * 8 + (size_t)(ks > 1 ? ks - 1 : 0) * mt * 32 * 8 * 4;
}

__global__ void k_restrict_tc(cplx<float>* __restrict__ out, const cplx<float>* __restrict__ in,
                              const __half2* __restrict__ P, const float* __restrict__ pscale, Geom gf, Geom gc,
                              bool fine, int n, int N, int nrhs, size_t in_rstride, size_t pstride,
                              size_t out_rstride, size_t out_site_stride, int ks) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned smax[RT_R];
  __shared__ float sscale[RT_R];
  unsigned* sP = reinterpret_cast<unsigned*>(smem);                       // [N][RT_PS] half2 words
  uint2* sX = reinterpret_cast<uint2*>(smem + (size_t)N * RT_PS * 4);     // [RT_R][RT_XS] float2, then {hi, lo}
  float* sRed = reinterpret_cast<float*>(smem + (size_t)N * RT_PS * 4 + (size_t)RT_R * RT_XS * 8);
  const int agg = blockIdx.x;
  const int r0 = blockIdx.y * RT_R;
  const int nr = min(RT_R, nrhs - r0);
  const int tid = threadIdx.x, nth = blockDim.x;
  const int V = gf.V, h = n / 2;
  const int K = gf.vA * h;
  const int mt_n = (2 * N + 15) / 16;
  const int warp = tid >> 5, lane = tid & 31;
  const int mtile = warp % mt_n, kq = warp / mt_n;
  const int gq = lane >> 2, tq = lane & 3;
  const int nt = nr > 8 ? 2 : 1;
  const int ja = mtile * 8 + (gq >> 1), jb = ja + 4;
  const bool imrow = (gq & 1) != 0;
  int c0[4];
  geom_coords(gf, agg * gf.vA, c0);
  const int cs = coarse_site_of(gf, gc, c0);
  for (int s = 0; s < 2; ++s) {
    float tot[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
    for (int k0 = 0; k0 < K; k0 += RT_KCH) {
      const int kc = min(RT_KCH, K - k0);
      if (tid < RT_R) smax[tid] = 0u;
      // P chunk: word (j, k) = P_j at the k-th (site, component) of chirality s, zero beyond
      for (int e = tid; e < N * RT_KCH; e += nth) {
        const int j = e / RT_KCH, k = e - j * RT_KCH;
        unsigned w = 0u;
        if (k < kc) {
          const int kk = k0 + k, xl = kk / h, f = s * h + (kk - xl * h);
          const __half2 p = P[(size_t)j * pstride + faddr(fine, V, n, agg * gf.vA + xl, f)];
          w = *reinterpret_cast<const unsigned*>(&p);
        }
        sP[j * RT_PS + k] = w;
      }
      __syncthreads();
      // the chunk of every column, its max |Re|, |Im| reduced per warp (shuffles), one atomic per warp
      for (int r = 0; r < RT_R; ++r) {
        float m = 0.f;
        float2* dst = reinterpret_cast<float2*>(sX) + (size_t)r * RT_XS;
        for (int k = tid; k < RT_KCH; k += nth) {
          float2 v = make_float2(0.f, 0.f);
          if (r < nr && k < kc) {
            const int kk = k0 + k, xl = kk / h, f = s * h + (kk - xl * h);
            const cplx<float> x = in[(size_t)(r0 + r) * in_rstride + faddr(fine, V, n, agg * gf.vA + xl, f)];
            v = make_float2(x.re, x.im);
            m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
          }
          dst[k] = v;
        }
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
        if ((tid & 31) == 0 && m > 0.f) atomicMax(&smax[r], __float_as_uint(m));
      }
      __syncthreads();
      if (tid < RT_R) {
        const float m = __uint_as_float(smax[tid]);
        int ex = 0;
        frexpf(m, &ex);
        sscale[tid] = m > 0.f ? ldexpf(1.f, ex) : 1.f;
      }
      __syncthreads();
      for (int r = 0; r < RT_R; ++r) {
        const float inv = 1.f / sscale[r];
        uint2* row = sX + (size_t)r * RT_XS;
        for (int k = tid; k < RT_KCH; k += nth) {
          const float2 v = reinterpret_cast<float2*>(row)[k];
          const float xr = v.x * inv, xi = v.y * inv;
          const __half2 hi = __floats2half2_rn(xr, xi);
          const float2 hf = __half22float2(hi);
          const __half2 lo = __floats2half2_rn(xr - hf.x, xi - hf.y);
          uint2 u;
          u.x = *reinterpret_cast<const unsigned*>(&hi);
          u.y = *reinterpret_cast<const unsigned*>(&lo);
          row[k] = u;
        }
      }
      __syncthreads();
      // FP32 accumulators: hi products in four chains (k-tile mod 4), lo products in their own (the
      // tensor core's accumulation truncates; short chains keep its bias from adding up along K)
      float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
      float ach[4][2][4] = {};
      const int KT = (kc + 7) / 8;
      const int kt0 = (kq * KT) / ks, kt1 = ((kq + 1) * KT) / ks;
      // A word of conj(P)^T: (Re p, Im p) on a real-part row, (-Im p, Re p) on an imaginary-part row
      auto afrag = [&](int j, int k) -> unsigned {
        if (j >= N) return 0u;
        const unsigned w = sP[j * RT_PS + k];
        return imrow ? (__byte_perm(w, 0, 0x1032) ^ 0x00008000u) : w;
      };
      for (int kt = kt0; kt < kt1; ++kt) {
        const int k1 = kt * 8 + tq, k2 = k1 + 4;
        unsigned a[4];
        a[0] = afrag(ja, k1);
        a[1] = afrag(jb, k1);
        a[2] = afrag(ja, k2);
        a[3] = afrag(jb, k2);
        const int ch = kt & 3;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          if (q < nt) {
            const int r = q * 8 + gq;
            const uint2 x0 = sX[r * RT_XS + k1];
            const uint2 x1 = sX[r * RT_XS + k2];
#pragma unroll
            for (int c = 0; c < 4; ++c)
              if (c == ch) mma_16816(ach[c][q], a, x0.x, x1.x);
            mma_16816(acc[q], a, x0.y, x1.y);
          }
        }
      }
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int v = 0; v < 4; ++v)
          acc[q][v] = ((ach[0][q][v] + ach[1][q][v]) + (ach[2][q][v] + ach[3][q][v])) + acc[q][v];
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int v = 0; v < 4; ++v) tot[q][v] += sscale[q * 8 + 2 * tq + (v & 1)] * acc[q][v];
      __syncthreads();   // before the next chunk overwrites the staged data
    }
    // fixed-order reduction of the k shares, then out = pscale(A, s) * total
    if (ks > 1) {
      if (kq > 0) {
        float* dst = sRed + ((size_t)((kq - 1) * mt_n + mtile) * 32 + lane) * 8;
#pragma unroll
        for (int q = 0; q < 8; ++q) dst[q] = tot[q >> 2][q & 3];
      }
      __syncthreads();
      if (kq == 0)
        for (int sh = 1; sh < ks; ++sh) {
          const float* src = sRed + ((size_t)((sh - 1) * mt_n + mtile) * 32 + lane) * 8;
#pragma unroll
          for (int q = 0; q < 8; ++q) tot[q >> 2][q & 3] += src[q];
        }
    }
    if (kq == 0) {
      const float ps = pscale ? pscale[agg * 2 + s] : 1.f;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        if (q >= nt) continue;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int row = mtile * 16 + gq + (v >= 2 ? 8 : 0);
          const int col = q * 8 + 2 * tq + (v & 1);
          const int j = row >> 1;
          if (j < N && col < nr) {
            float* o = reinterpret_cast<float*>(out + (size_t)(r0 + col) * out_rstride + (size_t)cs * out_site_stride +
                                                (size_t)s * N + j);
            o[row & 1] = ps * tot[q][v];
          }
        }
      }
    }
    __syncthreads();   // sRed reuse by the next chirality
  }
}

// out(x, f)[r] = [out +] pscale(A, s) * sum_j P_j(x, f) in_r(A)[s N + j], every r of the batch
template <int NMAX>
__global__ void k_prolong_batch(cplx<float>* __restrict__ out, const cplx<float>* __restrict__ in,
                                const __half2* __restrict__ P, const float* __restrict__ pscale, Geom gf, Geom gc,
                                bool fine, int n, int N, int nrhs, size_t out_rstride, size_t in_rstride,
                                size_t pstride, bool accumulate) {
  extern __shared__ __align__(16) unsigned char smem[];
  cplx<float>* sc = reinterpret_cast<cplx<float>*>(smem);   // [nrhs][2N]
  const int agg = blockIdx.x;
  const int V = gf.V, h = n / 2;
  int c0[4];
  geom_coords(gf, agg * gf.vA, c0);
  const int cs = coarse_site_of(gf, gc, c0);
  for (int e = threadIdx.x; e < nrhs * 2 * N; e += blockDim.x) {
    const int r = e / (2 * N), q = e - r * 2 * N;
    sc[e] = in[(size_t)r * in_rstride + (size_t)cs * 2 * N + q];
  }
  __syncthreads();
  const int rows = gf.vA * n;
  for (int t = threadIdx.x; t < rows; t += blockDim.x) {
    // fine level: component-major rows (consecutive threads take consecutive sites of one f)
    int xl, f;
    if (fine) { f = t / gf.vA; xl = t - f * gf.vA; }
    else { xl = t / n; f = t - xl * n; }
    const int x = agg * gf.vA + xl;
    const int s = f < h ? 0 : 1;
    const size_t a = faddr(fine, V, n, x, f);
    cplx<float> p[NMAX];
#pragma unroll
    for (int j = 0; j < NMAX; ++j)
      if (j < N) {
        const float2 v = __half22float2(P[(size_t)j * pstride + a]);
        p[j] = cmk<float>(v.x, v.y);
      }
    const float ps = pscale ? pscale[agg * 2 + s] : 1.f;
    for (int r = 0; r < nrhs; ++r) {
      const cplx<float>* cr = sc + (size_t)r * 2 * N + s * N;
      cplx<float> acc = czero<float>();
#pragma unroll
      for (int j = 0; j < NMAX; ++j)
        if (j < N) cfma(acc, p[j], cr[j]);
      acc = ps * acc;
      cplx<float>* po = out + (size_t)r * out_rstride + a;
      *po = accumulate ? *po + acc : acc;
    }
  }
}

// the kernel's dynamic shared-memory limit (process-wide) only ever grows, under a lock
cudaError_t prepare_restrict_tc(size_t bytes) {
  static std::atomic<size_t> set_to{0};
  static std::mutex mu;
  if (set_to.load(std::memory_order_acquire) >= bytes) return cudaSuccess;
  std::lock_guard<std::mutex> lk(mu);
  if (set_to.load(std::memory_order_relaxed) >= bytes) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(k_restrict_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) set_to.store(bytes, std::memory_order_release);
  return e;
}

}  // namespace

namespace dd {

bool restrict_tc_fits(int N, int ks) {
  const int mt = (2 * N + 15) / 16;
  return N >= 1 && N <= 32 && ks >= 1 && ks <= 4 && 32 * mt * ks <= 1024 && rt_smem(N, ks) <= 200 * 1024;
}

cudaError_t restrict_tc(cplx<float>* out, const cplx<float>* in, const __half2* Ph, const float* pscale,
                        const Geom& gf, const Geom& gc, bool fine, int n, int N, int nrhs, size_t in_rstride,
                        size_t out_rstride, size_t out_site_stride, int ks, cudaStream_t st) {
  if (nrhs <= 0) return cudaSuccess;
  if (!Ph || !restrict_tc_fits(N, ks)) return cudaErrorInvalidValue;
  const size_t bytes = rt_smem(N, ks);
  const cudaError_t e = prepare_restrict_tc(bytes);
  if (e != cudaSuccess) return e;
  const int threads = 32 * ((2 * N + 15) / 16) * ks;
  count_launch();
  k_restrict_tc<<<dim3(gf.nAgg, (nrhs + RT_R - 1) / RT_R), threads, bytes, st>>>(
      out, in, Ph, pscale, gf, gc, fine, n, N, nrhs, in_rstride, (size_t)gf.V * n, out_rstride,
      out_site_stride, ks);
  return cudaPeekAtLastError();
}

cudaError_t prolong_batch(cplx<float>* out, const cplx<float>* in, const __half2* Ph, const float* pscale,
                          const Geom& gf, const Geom& gc, bool fine, int n, int N, int nrhs, size_t out_rstride,
                          size_t in_rstride, bool accumulate, cudaStream_t st) {
  if (nrhs <= 0) return cudaSuccess;
  if (!Ph || N > 32) return cudaErrorInvalidValue;
  const size_t bytes = (size_t)nrhs * 2 * N * sizeof(cplx<float>);
  if (bytes > 48 * 1024) return cudaErrorInvalidValue;
  const size_t pstride = (size_t)gf.V * n;
  count_launch();
  const int threads = 256;
  if (N <= 8)
    k_prolong_batch<8><<<gf.nAgg, threads, bytes, st>>>(out, in, Ph, pscale, gf, gc, fine, n, N, nrhs, out_rstride,
                                                         in_rstride, pstride, accumulate);
  else if (N <= 16)
    k_prolong_batch<16><<<gf.nAgg, threads, bytes, st>>>(out, in, Ph, pscale, gf, gc, fine, n, N, nrhs, out_rstride,
                                                          in_rstride, pstride, accumulate);
  else if (N <= 24)
    k_prolong_batch<24><<<gf.nAgg, threads, bytes, st>>>(out, in, Ph, pscale, gf, gc, fine, n, N, nrhs, out_rstride,
                                                          in_rstride, pstride, accumulate);
  else
    k_prolong_batch<32><<<gf.nAgg, threads, bytes, st>>>(out, in, Ph, pscale, gf, gc, fine, n, N, nrhs, out_rstride,
                                                          in_rstride, pstride, accumulate);
  return cudaPeekAtLastError();
}

}  // namespace dd
