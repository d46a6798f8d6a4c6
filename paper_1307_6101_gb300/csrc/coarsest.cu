// Coarsest-level solve (Sec. 3 of the paper: odd-even preconditioned GMRES to
// relative accuracy epsilon) as one persistent kernel per right-hand side on a
// thread-block cluster.
//
// With D = [[S_ee, D_eo], [D_oe, S_oo]] and S_oo inverted at setup, GMRES(m)
// runs on Dhat = S_ee - D_eo S_oo^{-1} D_oe for bhat_e = b_e - D_eo S_oo^{-1} b_o;
// afterwards z_o = S_oo^{-1} (b_o - D_oe z_e).  CTA q of the cluster owns a
// contiguous slice of the even sites and of the odd sites.  It keeps its rows
// of the Krylov basis in shared memory; neighbour values are read from the
// owning CTA's shared memory (distributed shared memory), dot products are
// summed from per-CTA partials in rank order (identical in every CTA), and the
// Givens updates are computed redundantly by every CTA, so no CTA waits on a
// broadcast.  Cluster barriers separate the phases.  All loops are bounded by
// max_cycles * m.  Stopping rules are those of the host-driven solver: |g_{j+1}|
// <= tol ||bhat|| inside a cycle, the recomputed residual between cycles.
//
// Resident variant (NR > 0: FP32 arithmetic on FP16 blocks, one even and one odd
// site per CTA): the operator does not change during the solve, so each CTA
// loads it once -- the rows of its odd site's 8 hop blocks into registers (one
// row per thread), its even site's 9 blocks and its odd site's self inverse into
// shared memory by bulk copies -- and every GMRES step then reads the operator
// from registers and shared memory instead of L2.
#include <cooperative_groups.h>

#include "common.cuh"
#include "kernels.h"
#include "tma.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int MAXM = 64;
constexpr int RES_NR = 56;   // largest coarse dof count of the resident variant (rows held in registers)

DD_HD size_t bidx(int site, int k, int n, int i, int j) { return (((size_t)site * 9 + k) * n + j) * n + i; }

template <typename T>
struct Smem {
  cplx<T>* Vb;     // [m+1][ne_per*n] Krylov basis rows of the own even sites
  cplx<T>* xv;     // [ne_per*n] solution (even)
  cplx<T>* rv;     // [ne_per*n] residual / bhat
  cplx<T>* wv;     // [ne_per*n] new direction
  cplx<T>* be;     // [ne_per*n] b on the own even sites
  cplx<T>* bo;     // [no_per*n] b on the own odd sites
  cplx<T>* tv;     // [no_per*n] S_oo^{-1}(...) on the own odd sites
  cplx<T>* xs;     // [9][n] gathered neighbour vectors
  cplx<T>* part;   // [9][n] partial rows
  cplx<T>* us;     // [n]
  cplx<T>* red;    // [3][CL][MAXM] dot-product partials (read from rank 0)
  cplx<T>* H;      // [m+1][m]
  cplx<T>* g;      // [m+1]
  cplx<T>* sn;     // [m]
  cplx<T>* y;      // [m]
  cplx<T>* hsum;   // [MAXM] reduced dots of the current pass
  cplx<T>* htot;   // [MAXM] sum of both CGS passes
  T* cs;           // [m]
  T* scal;         // [8] broadcast scalars inside the CTA
  // resident variant only
  __half2* eblk;   // [9][n][n] blocks of the own even site
  cplx<T>* oinv;   // [n][n] self inverse of the own odd site
  unsigned long long* bar;
};

template <typename T>
__device__ Smem<T> carve(unsigned char* base, int m, int nep, int nop, int n, int CL) {
  // layout must match smem_bytes()
  Smem<T> s;
  cplx<T>* p = reinterpret_cast<cplx<T>*>(base);
  s.Vb = p; p += (size_t)(m + 1) * nep * n;
  s.xv = p; p += (size_t)nep * n;
  s.rv = p; p += (size_t)nep * n;
  s.wv = p; p += (size_t)nep * n;
  s.be = p; p += (size_t)nep * n;
  s.bo = p; p += (size_t)nop * n;
  s.tv = p; p += (size_t)nop * n;
  s.xs = p; p += (size_t)9 * n;
  s.part = p; p += (size_t)9 * n;
  s.us = p; p += (size_t)n;
  s.red = p; p += (size_t)3 * CL * MAXM;
  s.H = p; p += (size_t)(m + 1) * m;
  s.g = p; p += (size_t)(m + 1);
  s.sn = p; p += (size_t)m;
  s.y = p; p += (size_t)m;
  s.hsum = p; p += (size_t)MAXM;
  s.htot = p; p += (size_t)MAXM;
  T* q = reinterpret_cast<T*>(p);
  s.cs = q; q += m;
  s.scal = q;
  q += 8;
  uintptr_t a = (reinterpret_cast<uintptr_t>(q) + 15) & ~uintptr_t(15);
  s.eblk = reinterpret_cast<__half2*>(a);
  a += (size_t)9 * n * n * sizeof(__half2);
  s.oinv = reinterpret_cast<cplx<T>*>(a);
  a += (size_t)n * n * sizeof(cplx<T>);
  s.bar = reinterpret_cast<unsigned long long*>(a);
  return s;
}

template <typename T>
struct Ctx {
  const cplx<T>* blk;
  const __half2* blkh;     // FP16 blocks (FP32 compute only) or null
  const float* bscale;     // per-site scale of blkh
  const cplx<T>* inv;
  const int* even;
  const int* odd;
  const int* nbr_e_of_o;   // [n_o][8] even-list index of neighbour k (k<4: +mu, k>=4: -mu)
  const int* nbr_o_of_e;   // [n_e][8]
  int* err;                // bounded-wait error flag
  int n_e, n_o, nep, nop, n, CL, rank;
};

// operator rows held by one thread of the resident variant
template <int NR>
struct RegRows {
  __half2 r[NR > 0 ? NR : 1];
};

// acc += sum_j M(site, k)[i][j] xv[j] from the compute-precision or the FP16 blocks
template <typename T>
__device__ __forceinline__ cplx<T> block_row(const Ctx<T>& cx, int site, int k, int i, const cplx<T>* xv) {
  const int n = cx.n;
  // two accumulators (even and odd columns): two independent chains of fused multiply-adds
  cplx<T> acc = czero<T>(), acc1 = czero<T>();
  if constexpr (sizeof(T) == 4) {
    if (cx.blkh) {
      const __half2* M = cx.blkh + bidx(site, k, n, i, 0);
      int j = 0;
#pragma unroll 4
      for (; j + 1 < n; j += 2) {
        cfma(acc, ld_cplx(M, (size_t)j * n), xv[j]);
        cfma(acc1, ld_cplx(M, (size_t)(j + 1) * n), xv[j + 1]);
      }
      if (j < n) cfma(acc, ld_cplx(M, (size_t)j * n), xv[j]);
      return T(cx.bscale[site]) * (acc + acc1);
    }
  }
  const cplx<T>* M = cx.blk + bidx(site, k, n, i, 0);
  int j = 0;
#pragma unroll 4
  for (; j + 1 < n; j += 2) {
    cfma(acc, M[(size_t)j * n], xv[j]);
    cfma(acc1, M[(size_t)(j + 1) * n], xv[j + 1]);
  }
  if (j < n) cfma(acc, M[(size_t)j * n], xv[j]);
  return acc + acc1;
}

// t(own odd) = S^{-1} ( a*bo + c * sum_k D_k(o) v(even nbr_k) ), v read from the owners' array `src`
template <typename T, int NR>
__device__ void odd_phase(const Ctx<T>& cx, const Smem<T>& s, cg::cluster_group& cluster, cplx<T>* src, T a, T c,
                          const RegRows<NR>& orow) {
  const int n = cx.n;
  if constexpr (NR > 0) {
    // one odd site per CTA; hop rows in registers, self inverse in shared memory
    const int o = cx.rank;
    if (o >= cx.n_o) return;   // uniform in the CTA
    const int site = cx.odd[o];
    if (c != T(0)) {
      for (int t = threadIdx.x; t < 8 * n; t += blockDim.x) {
        const int k = t / n, j = t - k * n;
        const int nb = cx.nbr_e_of_o[o * 8 + k];
        const cplx<T>* rem = cluster.map_shared_rank(src, nb / cx.nep);
        s.xs[t] = rem[(nb % cx.nep) * n + j];
      }
    }
    __syncthreads();
    {
      const int k = threadIdx.x / n, i = threadIdx.x - (threadIdx.x / n) * n;
      if (k < 8) {
        cplx<T> acc = czero<T>();
        if (c != T(0)) {
          const cplx<T>* xv = s.xs + k * n;
#pragma unroll
          for (int j = 0; j < NR; ++j)
            if (j < n) {
              const float2 f = __half22float2(orow.r[j]);
              cfma(acc, cmk<T>(f.x, f.y), xv[j]);
            }
          acc = T(cx.bscale[site]) * acc;
        }
        s.part[k * n + i] = acc;
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      cplx<T> u = czero<T>();
#pragma unroll
      for (int q = 0; q < 8; ++q) u = u + s.part[q * n + i];
      u = c * u;
      if (a != T(0)) u = u + a * s.bo[i];
      s.us[i] = u;
    }
    __syncthreads();
    // t = S^{-1} u: 8 lanes per row, each a strided share of the columns, summed by shuffles
    // (the loop runs to a multiple of 32 so that whole warps take part in the shuffles)
    for (int t = threadIdx.x; t < ((8 * n + 31) & ~31); t += blockDim.x) {
      const int i = t >> 3, q = t & 7;
      cplx<T> acc = czero<T>();
      if (i < n)
        for (int j = q; j < n; j += 8) cfma(acc, s.oinv[(size_t)j * n + i], s.us[j]);
#pragma unroll
      for (int off = 4; off >= 1; off >>= 1) {
        acc.re += __shfl_xor_sync(0xffffffffu, acc.re, off);
        acc.im += __shfl_xor_sync(0xffffffffu, acc.im, off);
      }
      if (q == 0 && i < n) s.tv[i] = acc;
    }
    __syncthreads();
  } else {
  for (int so = 0; so < cx.nop; ++so) {
    const int o = cx.rank * cx.nop + so;
    if (o >= cx.n_o) break;   // uniform in the CTA
    const int site = cx.odd[o];
    if (c != T(0)) {
      for (int t = threadIdx.x; t < 8 * n; t += blockDim.x) {
        const int k = t / n, j = t - k * n;
        const int nb = cx.nbr_e_of_o[o * 8 + k];
        const cplx<T>* rem = cluster.map_shared_rank(src, nb / cx.nep);
        s.xs[t] = rem[(nb % cx.nep) * n + j];
      }
    }
    __syncthreads();
    {
      const int k = threadIdx.x / n, i = threadIdx.x - (threadIdx.x / n) * n;
      if (k < 8) {
        cplx<T> acc = czero<T>();
        if (c != T(0)) acc = block_row(cx, site, 1 + k, i, s.xs + k * n);
        s.part[k * n + i] = acc;
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      cplx<T> u = czero<T>();
#pragma unroll
      for (int q = 0; q < 8; ++q) u = u + s.part[q * n + i];
      u = c * u;
      if (a != T(0)) u = u + a * s.bo[so * n + i];
      s.us[i] = u;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      cplx<T> acc = czero<T>();
      const cplx<T>* Mi = cx.inv + ((size_t)site * n) * n + i;
#pragma unroll 8
      for (int j = 0; j < n; ++j) cfma(acc, Mi[(size_t)j * n], s.us[j]);
      s.tv[so * n + i] = acc;
    }
    __syncthreads();
  }
  }
}

// dst(own even) = a*be + sc * S(e) xloc(e) + c * sum_k D_k(e) t(odd nbr_k)  (t read from the owners' tv)
template <typename T, int NR>
__device__ void even_phase(const Ctx<T>& cx, const Smem<T>& s, cg::cluster_group& cluster, const cplx<T>* xloc,
                           cplx<T>* dst, T a, T sc, T c) {
  const int n = cx.n;
  for (int se = 0; se < cx.nep; ++se) {
    const int e = cx.rank * cx.nep + se;
    if (e >= cx.n_e) break;
    const int site = cx.even[e];
    for (int t = threadIdx.x; t < 9 * n; t += blockDim.x) {
      const int k = t / n, j = t - k * n;
      cplx<T> v = czero<T>();
      if (k == 0) {
        if (sc != T(0)) v = xloc[se * n + j];
      } else if (c != T(0)) {
        const int nb = cx.nbr_o_of_e[e * 8 + k - 1];
        const cplx<T>* rem = cluster.map_shared_rank(s.tv, nb / cx.nop);
        v = rem[(nb % cx.nop) * n + j];
      }
      s.xs[t] = v;
    }
    __syncthreads();
    {
      const int k = threadIdx.x / n, i = threadIdx.x - (threadIdx.x / n) * n;
      if (k < 9) {
        cplx<T> acc = czero<T>();
        const T w = k == 0 ? sc : c;
        if (w != T(0)) {
          if constexpr (NR > 0) {   // the own even site's blocks are in shared memory
            const __half2* M = s.eblk + (size_t)k * n * n + i;
            const cplx<T>* xv = s.xs + k * n;
            cplx<T> acc1 = czero<T>();
            int j = 0;
#pragma unroll 4
            for (; j + 1 < n; j += 2) {
              cfma(acc, ld_cplx(M, (size_t)j * n), xv[j]);
              cfma(acc1, ld_cplx(M, (size_t)(j + 1) * n), xv[j + 1]);
            }
            if (j < n) cfma(acc, ld_cplx(M, (size_t)j * n), xv[j]);
            acc = T(cx.bscale[site]) * (acc + acc1);
          } else {
            acc = block_row(cx, site, k, i, s.xs + k * n);
          }
        }
        s.part[k * n + i] = w * acc;
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      cplx<T> v = czero<T>();
#pragma unroll
      for (int q = 0; q < 9; ++q) v = v + s.part[q * n + i];
      if (a != T(0)) v = v + a * s.be[se * n + i];
      dst[se * n + i] = v;
    }
    __syncthreads();
  }
}

// CTA-local sum of a complex value per thread; result in s.scal[0..1] (valid after return)
template <typename T>
__device__ void cta_sum_c(T re, T im, const Smem<T>& s, cplx<T>* buf) {
  for (int off = 16; off >= 1; off >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, off);
    im += __shfl_xor_sync(0xffffffffu, im, off);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) buf[warp] = cmk<T>(re, im);
  __syncthreads();
  if (threadIdx.x == 0) {
    cplx<T> t = czero<T>();
    for (int w = 0; w < nw; ++w) t = t + buf[w];
    s.scal[0] = t.re;
    s.scal[1] = t.im;
  }
  __syncthreads();
}

// h[d] = sum over all CTAs of conj(V_d) . w for d <= j and, with with_norm, h[j+1] = ||w||^2.
// Groups of 16 lanes own one d each and reduce with shuffles (fixed order); lane q of the
// group then writes the CTA's partial into CTA q's buffer `slot`, so after the barrier
// every CTA sums its own copy in rank order (identical in every CTA, local reads only).
template <typename T>
__device__ void cluster_dots(const Ctx<T>& cx, const Smem<T>& s, cg::cluster_group& cluster, const cplx<T>* w,
                             int j, int slot, int len, bool with_norm) {
  cplx<T>* red = s.red + (size_t)slot * cx.CL * MAXM;
  const int G = 16;
  const int grp = threadIdx.x / G, l = threadIdx.x % G, ngrp = blockDim.x / G;
  const int dmax = with_norm ? j + 1 : j;
  for (int d0 = 0; d0 <= dmax; d0 += ngrp) {
    const int d = d0 + grp;
    T re = T(0), im = T(0);
    if (d <= j) {
      const cplx<T>* v = s.Vb + (size_t)d * len;
      for (int e = l; e < len; e += G) {
        const cplx<T> t = cdotc(v[e], w[e]);
        re += t.re;
        im += t.im;
      }
    } else if (d == dmax) {
      for (int e = l; e < len; e += G) re += cnorm2(w[e]);
    }
    for (int off = G / 2; off >= 1; off >>= 1) {
      re += __shfl_xor_sync(0xffffffffu, re, off);
      im += __shfl_xor_sync(0xffffffffu, im, off);
    }
    if (d <= dmax && l < cx.CL) cluster.map_shared_rank(red, l)[cx.rank * MAXM + d] = cmk<T>(re, im);
  }
  cluster.sync();
  for (int d = threadIdx.x; d <= dmax; d += blockDim.x) {
    cplx<T> t = czero<T>();
    for (int q = 0; q < cx.CL; ++q) t = t + red[q * MAXM + d];
    s.hsum[d] = t;
  }
  __syncthreads();
}

// ||w||^2 over the cluster (rank-ordered; every CTA sums its own copy of the partials)
template <typename T>
__device__ T cluster_norm2(const Ctx<T>& cx, const Smem<T>& s, cg::cluster_group& cluster, const cplx<T>* w, int len) {
  cplx<T>* red = s.red + (size_t)2 * cx.CL * MAXM;
  T a = T(0);
  for (int e = threadIdx.x; e < len; e += blockDim.x) a += cnorm2(w[e]);
  cta_sum_c(a, T(0), s, s.part);
  if (threadIdx.x < cx.CL) cluster.map_shared_rank(red, threadIdx.x)[cx.rank * MAXM] = cmk<T>(s.scal[0], T(0));
  cluster.sync();
  if (threadIdx.x == 0) {
    T t = T(0);
    for (int q = 0; q < cx.CL; ++q) t += red[q * MAXM].re;
    s.scal[4] = t;
  }
  __syncthreads();
  return s.scal[4];
}

template <typename T, int NR>
__global__ void __launch_bounds__(512, 1) k_coarsest_cluster(Ctx<T> cx0, const cplx<T>* __restrict__ b, cplx<T>* __restrict__ x, size_t rstride,
                                   int m, int max_cycles, double tol, int* iters) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cg::cluster_group cluster = cg::this_cluster();
  Ctx<T> cx = cx0;
  cx.rank = (int)cluster.block_rank();
  const int n = cx.n;
  const int len = cx.nep * n;
  Smem<T> s = carve<T>(smem_raw, m, cx.nep, cx.nop, n, cx.CL);
  const cplx<T>* pb = b + (size_t)blockIdx.y * rstride;
  cplx<T>* px = x + (size_t)blockIdx.y * rstride;
  RegRows<NR> orow;
  int staged = 1;
  if constexpr (NR > 0) {
    // stage the own sites' operator: even site's 9 blocks and odd site's self inverse
    // (shared memory, bulk copies), odd site's 8 hop rows (registers)
    const int e = cx.rank, o = cx.rank;
    if (threadIdx.x == 0) {
      mbar_init(s.bar, 1);
      const unsigned be_bytes = (unsigned)(9 * n * n * sizeof(__half2));
      const unsigned bi_bytes = (unsigned)(n * n * sizeof(cplx<T>));
      mbar_arrive_expect_tx(s.bar, (e < cx.n_e ? be_bytes : 0u) + (o < cx.n_o ? bi_bytes : 0u));
      if (e < cx.n_e) bulk_g2s(s.eblk, cx.blkh + (size_t)cx.even[e] * 9 * n * n, be_bytes, s.bar);
      if (o < cx.n_o) bulk_g2s(s.oinv, cx.inv + (size_t)cx.odd[o] * n * n, bi_bytes, s.bar);
    }
    const int k = threadIdx.x / n, i = threadIdx.x - (threadIdx.x / n) * n;
    if (k < 8 && o < cx.n_o) {
      const __half2* M = cx.blkh + bidx(cx.odd[o], 1 + k, n, i, 0);
#pragma unroll
      for (int j = 0; j < NR; ++j) orow.r[j] = j < n ? M[(size_t)j * n] : __half2();
    }
    __syncthreads();
    staged = __syncthreads_and(mbar_wait_bounded(s.bar, 0) ? 1 : 0);
    if (!staged && threadIdx.x == 0) atomicExch(cx.err, 2);
  }
  // own b, zero x
  for (int t = threadIdx.x; t < len; t += blockDim.x) {
    const int e = cx.rank * cx.nep + t / n;
    s.be[t] = e < cx.n_e ? pb[(size_t)cx.even[e] * n + t % n] : czero<T>();
    s.xv[t] = czero<T>();
  }
  for (int t = threadIdx.x; t < cx.nop * n; t += blockDim.x) {
    const int o = cx.rank * cx.nop + t / n;
    s.bo[t] = o < cx.n_o ? pb[(size_t)cx.odd[o] * n + t % n] : czero<T>();
  }
  __syncthreads();
  // bhat_e = b_e - D_eo S_oo^{-1} b_o  -> rv
  odd_phase<T, NR>(cx, s, cluster, s.xv, T(1), T(0), orow);
  cluster.sync();
  even_phase<T, NR>(cx, s, cluster, s.xv, s.rv, T(1), T(0), T(-1));
  const T bnorm = sqrt(cluster_norm2<T>(cx, s, cluster, s.rv, len));
  const T target = (T)tol * bnorm;
  // keep bhat: be <- rv (be is not needed any more)
  for (int t = threadIdx.x; t < len; t += blockDim.x) s.be[t] = s.rv[t];
  __syncthreads();
  T beta = bnorm;
  int total = 0;
  for (int cycle = 0; cycle < max_cycles; ++cycle) {
    if (!(beta > target)) break;   // converged (or zero rhs): uniform in the cluster
    const T iv = T(1) / beta;
    for (int t = threadIdx.x; t < len; t += blockDim.x) s.Vb[t] = iv * s.rv[t];
    if (threadIdx.x == 0) {
      for (int k = 0; k <= m; ++k) s.g[k] = czero<T>();
      s.g[0] = cmk<T>(beta, T(0));
    }
    cluster.sync();
    int kk = 0;
    for (int j = 0; j < m; ++j) {
      cplx<T>* vj = s.Vb + (size_t)j * len;
      // w = Dhat v_j
      odd_phase<T, NR>(cx, s, cluster, vj, T(0), T(1), orow);
      cluster.sync();
      even_phase<T, NR>(cx, s, cluster, vj, s.wv, T(0), T(1), T(-1));
      // CGS2; the second pass also sums ||w'||^2, and ||w''||^2 = ||w'||^2 - sum_d |h2_d|^2
      // (w'' = w' - V h2 with h2 = V^+ w' and V orthonormal), which saves a reduction
      for (int pass = 0; pass < 2; ++pass) {
        cluster_dots<T>(cx, s, cluster, s.wv, j, pass, len, pass == 1);
        for (int d = threadIdx.x; d <= j; d += blockDim.x) s.htot[d] = pass == 0 ? s.hsum[d] : s.htot[d] + s.hsum[d];
        if (pass == 1 && threadIdx.x < 32) {   // sum_d |h2_d|^2 by warp 0 (strided partials, shuffle tree)
          T h2 = T(0);
          for (int d = threadIdx.x; d <= j; d += 32) h2 += cnorm2(s.hsum[d]);
          for (int off = 16; off >= 1; off >>= 1) h2 += __shfl_xor_sync(0xffffffffu, h2, off);
          if (threadIdx.x == 0) s.scal[5] = s.hsum[j + 1].re - h2;
        }
        // w -= sum_d h_d V_d: 8 lanes per element, each a strided share of d, summed by shuffles
        // (the loop runs to a multiple of 32 so that whole warps take part in the shuffles)
        for (int t = threadIdx.x; t < ((8 * len + 31) & ~31); t += blockDim.x) {
          const int e = t >> 3, q = t & 7;
          cplx<T> acc = czero<T>();
          if (e < len)
            for (int d = q; d <= j; d += 8) cfma(acc, s.hsum[d], s.Vb[(size_t)d * len + e]);
#pragma unroll
          for (int off = 4; off >= 1; off >>= 1) {
            acc.re += __shfl_xor_sync(0xffffffffu, acc.re, off);
            acc.im += __shfl_xor_sync(0xffffffffu, acc.im, off);
          }
          if (q == 0 && e < len) s.wv[e] = s.wv[e] - acc;
        }
        __syncthreads();
      }
      const T hn = sqrt(s.scal[5] > T(0) ? s.scal[5] : T(0));
      // Givens update, identical in every CTA
      if (threadIdx.x == 0) {
        // the previous rotations applied to the new column, the running entry carried in registers
        cplx<T> cur = s.htot[0];
        for (int i = 0; i < j; ++i) {
          const cplx<T> nx = s.htot[i + 1];
          const cplx<T> t = s.cs[i] * cur + s.sn[i] * nx;
          cur = s.cs[i] * nx - cconj(s.sn[i]) * cur;
          s.H[(size_t)i * m + j] = t;
        }
        cplx<T> h[2] = {cur, cmk<T>(hn, T(0))};   // entries j and j + 1
        const T aa = sqrt(cnorm2(h[0])), bb = sqrt(cnorm2(h[1]));
        const T rr = sqrt(aa * aa + bb * bb);
        T c;
        cplx<T> sg;
        if (rr == T(0)) { c = T(1); sg = czero<T>(); }
        else if (aa == T(0)) { c = T(0); sg = bb == T(0) ? cmk<T>(T(1), T(0)) : cmk<T>(h[1].re / bb, -h[1].im / bb); }
        else {
          c = aa / rr;
          const cplx<T> ph = cmk<T>(h[0].re / aa, h[0].im / aa);
          sg = (T(1) / rr) * (ph * cconj(h[1]));
        }
        s.cs[j] = c;
        s.sn[j] = sg;
        s.H[(size_t)j * m + j] = c * h[0] + sg * h[1];
        s.g[j + 1] = T(-1) * (cconj(sg) * s.g[j]);
        s.g[j] = c * s.g[j];
        const T est = sqrt(cnorm2(s.g[j + 1]));
        const int stop = (est <= target || hn == T(0) || j + 1 == m) ? 1 : 0;
        s.scal[2] = stop ? T(1) : T(0);
        s.scal[3] = hn > T(0) ? T(1) / hn : T(0);
      }
      __syncthreads();
      const bool stop = s.scal[2] != T(0);
      const T ivn = s.scal[3];
      kk = j + 1;
      if (!stop) {
        cplx<T>* vn = s.Vb + (size_t)(j + 1) * len;
        for (int e = threadIdx.x; e < len; e += blockDim.x) vn[e] = ivn * s.wv[e];
      }
      cluster.sync();
      if (stop) break;
    }
    total += kk;
    // y = R^{-1} g, x += V y
    if (threadIdx.x == 0) {
      for (int i = kk - 1; i >= 0; --i) {
        cplx<T> t = s.g[i];
        for (int l = i + 1; l < kk; ++l) t = t - s.H[(size_t)i * m + l] * s.y[l];
        const cplx<T> d = s.H[(size_t)i * m + i];
        const T dn = cnorm2(d);
        s.y[i] = dn > T(0) ? (T(1) / dn) * (t * cconj(d)) : czero<T>();
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < len; e += blockDim.x) {
      cplx<T> xe = s.xv[e];
      for (int i = 0; i < kk; ++i) xe = xe + s.y[i] * s.Vb[(size_t)i * len + e];
      s.xv[e] = xe;
    }
    cluster.sync();
    if (cycle + 1 == max_cycles) break;
    // true residual r = bhat - Dhat x
    odd_phase<T, NR>(cx, s, cluster, s.xv, T(0), T(1), orow);
    cluster.sync();
    even_phase<T, NR>(cx, s, cluster, s.xv, s.rv, T(1), T(-1), T(1));   // uses be = bhat as b
    beta = sqrt(cluster_norm2<T>(cx, s, cluster, s.rv, len));
  }
  // z_o = S_oo^{-1} (b_o - D_oe x_e); write x
  cluster.sync();
  odd_phase<T, NR>(cx, s, cluster, s.xv, T(1), T(-1), orow);
  for (int t = threadIdx.x; staged && t < len; t += blockDim.x) {
    const int e = cx.rank * cx.nep + t / n;
    if (e < cx.n_e) px[(size_t)cx.even[e] * n + t % n] = s.xv[t];
  }
  for (int t = threadIdx.x; staged && t < cx.nop * n; t += blockDim.x) {
    const int o = cx.rank * cx.nop + t / n;
    if (o < cx.n_o) px[(size_t)cx.odd[o] * n + t % n] = s.tv[t];
  }
  if constexpr (NR > 0)
    if (!staged && threadIdx.x == 0) mbar_wait_bounded(s.bar, 0);   // no copy in flight at exit
  if (cx.rank == 0 && threadIdx.x == 0 && iters) atomicAdd(iters, total);
  cluster.sync();   // no CTA exits while others may still read its shared memory
}

template <typename T>
size_t smem_bytes(int m, int nep, int nop, int n, int CL, bool resident) {
  size_t c = (size_t)(m + 1) * nep * n + 4 * (size_t)nep * n + 2 * (size_t)nop * n + 18 * (size_t)n + n +
             3 * (size_t)CL * MAXM + (size_t)(m + 1) * m + (m + 1) + 2 * (size_t)m + 2 * MAXM;
  size_t b = c * sizeof(cplx<T>) + (m + 8) * sizeof(T) + 16;
  if (resident) b += (size_t)9 * n * n * sizeof(__half2) + (size_t)n * n * sizeof(cplx<T>) + 16;
  return b + 64;
}

}  // namespace

namespace dd {

// the dynamic shared-memory limit is a process-wide attribute of the kernel: raised to the device
// maximum, so that hierarchies set up later with a smaller coarsest level do not lower it
template <typename T, int NR>
bool cluster_fits(int CL, int threads, size_t sm) {
  if (cudaFuncSetAttribute(k_coarsest_cluster<T, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024) !=
      cudaSuccess) {
    cudaGetLastError();
    cudaFuncSetAttribute(k_coarsest_cluster<T, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  }
  if (CL > 8) cudaFuncSetAttribute(k_coarsest_cluster<T, NR>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(CL, 1, 1);
  cfg.blockDim = dim3(threads, 1, 1);
  cfg.dynamicSmemBytes = sm;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nclusters = 0;
  if (cudaOccupancyMaxActiveClusters(&nclusters, k_coarsest_cluster<T, NR>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return nclusters >= 1;
}

// Chooses the cluster size (16 if the device can co-schedule it, else 8, 4, 2)
// and reports whether the cluster kernel can run this level (shared memory).
// For FP32 it also records whether the resident variant (FP16 blocks, one even
// and one odd site per CTA) fits.
template <typename T>
int coarsest_cluster_plan(const CoarsestPlanIn& in, CoarsestPlan* plan) {
  const int n_e = in.n_even, n_o = in.n_odd;
  for (int CL : {16, 8, 4, 2}) {
    if (CL > n_e || CL > n_o) continue;
    const int nep = (n_e + CL - 1) / CL, nop = (n_o + CL - 1) / CL;
    const size_t sm = smem_bytes<T>(in.m, nep, nop, in.n, CL, false);
    if (sm > 220 * 1024) continue;
    int threads = ((9 * in.n + 31) / 32) * 32;
    if (threads < 256) threads = 256;
    if (threads > 1024) return 0;
    if (!cluster_fits<T, 0>(CL, threads, sm)) continue;
    plan->CL = CL;
    plan->nep = nep;
    plan->nop = nop;
    plan->threads = threads;
    plan->smem = sm;
    plan->res_nr = 0;
    plan->res_smem = 0;
    if constexpr (sizeof(T) == 4) {
      const size_t smr = smem_bytes<T>(in.m, nep, nop, in.n, CL, true);
      if (nep == 1 && nop == 1 && in.n <= RES_NR && threads <= 512 && smr <= 227 * 1024 &&
          cluster_fits<T, RES_NR>(CL, threads, smr)) {
        plan->res_nr = RES_NR;
        plan->res_smem = smr;
      }
    }
    return 1;
  }
  return 0;
}

template <typename T>
cudaError_t coarsest_cluster_solve(cplx<T>* x, const cplx<T>* b, const CoarseOp<T>& op, const CoarsestPlan& plan,
                                   const CoarsestGeo& geo, int nrhs, size_t rstride, int m, int max_cycles, double tol,
                                   int* iters, cudaStream_t st) {
  Ctx<T> cx;
  cx.blk = op.blk;
  cx.blkh = op.blkh;
  cx.bscale = op.bscale;
  cx.inv = op.selfinv;
  cx.even = geo.even;
  cx.odd = geo.odd;
  cx.nbr_e_of_o = geo.nbr_e_of_o;
  cx.nbr_o_of_e = geo.nbr_o_of_e;
  cx.err = op.err;
  cx.n_e = geo.n_even;
  cx.n_o = geo.n_odd;
  cx.nep = plan.nep;
  cx.nop = plan.nop;
  cx.n = op.n;
  cx.CL = plan.CL;
  cx.rank = 0;
  const bool resident = sizeof(T) == 4 && op.blkh && plan.res_nr > 0;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = plan.CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(plan.CL, nrhs, 1);
  cfg.blockDim = dim3(plan.threads, 1, 1);
  cfg.dynamicSmemBytes = resident ? plan.res_smem : plan.smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  count_launch();
  if constexpr (sizeof(T) == 4)
    if (resident)
      return cudaLaunchKernelEx(&cfg, k_coarsest_cluster<T, RES_NR>, cx, b, x, rstride, m, max_cycles, tol, iters);
  return cudaLaunchKernelEx(&cfg, k_coarsest_cluster<T, 0>, cx, b, x, rstride, m, max_cycles, tol, iters);
}

#define INST(T)                                                                                                     \
  template int coarsest_cluster_plan<T>(const CoarsestPlanIn&, CoarsestPlan*);                                      \
  template cudaError_t coarsest_cluster_solve<T>(cplx<T>*, const cplx<T>*, const CoarseOp<T>&, const CoarsestPlan&,  \
                                                 const CoarsestGeo&, int, size_t, int, int, double, int*, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace dd
