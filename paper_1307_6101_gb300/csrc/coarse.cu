// Coarse-level kernels: the Galerkin operators D_{l+1} = P_l^+ D_l P_l are
// nearest-neighbour stencils of dense n x n complex blocks (Sec. 1, Sec. 2):
//   (D phi)(A) = S(A) phi(A) + sum_mu [ F_mu(A) phi(A + mu) + B_mu(A) phi(A - mu) ].
// Blocks are stored column-major per (site, k) with k = 0 self, 1..4 forward,
// 5..8 backward, so that the threads computing consecutive rows of one site
// read consecutive words.
#include <atomic>
#include <cooperative_groups.h>

#include "common.cuh"
#include "kernels.h"
#include "tma.cuh"

namespace cg = cooperative_groups;

namespace {

DD_HD size_t bidx(int site, int k, int n, int i, int j) { return (((size_t)site * 9 + k) * n + j) * n + i; }

template <typename T>
__device__ void cta_sum3(T& a, T& b, T& c, T* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  for (int off = 16; off >= 1; off >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, off);
    b += __shfl_xor_sync(0xffffffffu, b, off);
    c += __shfl_xor_sync(0xffffffffu, c, off);
  }
  if (lane == 0) { sh[3 * warp] = a; sh[3 * warp + 1] = b; sh[3 * warp + 2] = c; }
  __syncthreads();
  a = b = c = T(0);
  for (int w = 0; w < nw; ++w) { a += sh[3 * w]; b += sh[3 * w + 1]; c += sh[3 * w + 2]; }
  __syncthreads();
}

// (D phi)(A): one CTA per coarse site, one thread per (row i, block k); the
// neighbour vectors are staged in shared memory and the 9 partial rows are
// summed in shared memory.  Blocks are column-major, so the threads of one k
// read consecutive words for every column j.
template <typename T, bool RESID, typename BS>
__global__ void k_coarse_apply(cplx<T>* __restrict__ out, const cplx<T>* __restrict__ in,
                               const cplx<T>* __restrict__ bsrc, const BS* __restrict__ blk,
                               const float* __restrict__ bscale, Geom g, int n, size_t rstride, int sel, int sel_mu,
                               int in_chir) {
  extern __shared__ unsigned char smem_raw[];
  cplx<T>* xs = reinterpret_cast<cplx<T>*>(smem_raw);   // [9][n] neighbour vectors
  cplx<T>* part = xs + 9 * n;                           // [9][n] partial rows
  __shared__ int nbr[9];
  __shared__ int take[9];
  const int site = blockIdx.x;
  const size_t ro = (size_t)blockIdx.y * rstride;
  const cplx<T>* pin = in + ro;
  if (threadIdx.x < 9) {
    int c[4];
    geom_coords(g, site, c);
    const int k = threadIdx.x;
    int nb = site;
    bool tk = sel == SEL_FULL || sel == SEL_AGG_SELF;
    if (k > 0) {
      const int mu = (k - 1) % 4, dir = k <= 4 ? +1 : -1;
      nb = geom_neighbor(g, c, mu, dir);
      const bool internal = hop_internal(g, c, mu, dir, g.A);
      if (sel == SEL_FULL) tk = true;
      else if (sel == SEL_AGG_SELF) tk = internal;
      else if (sel == SEL_AGG_FWD) tk = dir > 0 && mu == sel_mu && !internal;
      else tk = dir < 0 && mu == sel_mu && !internal;
    }
    nbr[k] = nb;
    take[k] = tk;
  }
  __syncthreads();
  const int h = n / 2;
  for (int e = threadIdx.x; e < 9 * n; e += blockDim.x) {
    const int k = e / n, j = e % n;
    const bool keep = take[k] && (in_chir < 0 || (j < h) == (in_chir == 0));
    xs[e] = keep ? pin[(size_t)nbr[k] * n + j] : czero<T>();
  }
  __syncthreads();
  const int k = threadIdx.x / n, i = threadIdx.x % n;
  if (k < 9) {
    cplx<T> acc = czero<T>();
    if (take[k]) {
      const BS* M = blk + (((size_t)site * 9 + k) * n) * n + i;
      const cplx<T>* x = xs + k * n;
#pragma unroll 8
      for (int j = 0; j < n; ++j) cfma(acc, ld_cplx(M, (size_t)j * n), x[j]);
      if (bscale) acc = T(bscale[site]) * acc;
    }
    part[k * n + i] = acc;
  }
  __syncthreads();
  if (threadIdx.x < n) {
    cplx<T> y = czero<T>();
#pragma unroll
    for (int q = 0; q < 9; ++q) y = y + part[q * n + threadIdx.x];
    const size_t a = ro + (size_t)site * n + threadIdx.x;
    out[a] = RESID ? bsrc[a] - y : y;
  }
}

// Even-odd pieces of the coarsest solve (Sec. 3: odd-even preconditioned GMRES),
// with D = [[S_ee, D_eo], [D_oe, S_oo]] and the self blocks S inverted at setup.
// k_schur_odd: on every odd site A,  t(A) = S(A)^{-1} ( a*b(A) + c*(D_oe x)(A) )
//              (even entries of t are not written)
// k_schur_even: on every even site A, y(A) = a*b(A) + s*S(A) x(A) + c*(D_eo t)(A);
//              odd entries of y are set to zero.
template <typename T, typename BS>
__global__ void k_schur_odd(cplx<T>* __restrict__ t, const cplx<T>* __restrict__ x, const cplx<T>* __restrict__ b,
                            const BS* __restrict__ blk, const float* __restrict__ bscale,
                            const cplx<T>* __restrict__ inv,
                            const int* __restrict__ odd_sites, Geom g, int n, size_t rstride, double a, double c) {
  extern __shared__ unsigned char smem_raw[];
  cplx<T>* xs = reinterpret_cast<cplx<T>*>(smem_raw);   // [8][n]
  cplx<T>* part = xs + 8 * n;                           // [8][n]
  cplx<T>* u = part + 8 * n;                            // [n]
  __shared__ int nbr[8];
  const size_t ro = (size_t)blockIdx.y * rstride;
  const int site = odd_sites[blockIdx.x];
  if (threadIdx.x < 8) {
    int cc[4];
    geom_coords(g, site, cc);
    const int k = threadIdx.x;
    nbr[k] = geom_neighbor(g, cc, k % 4, k < 4 ? +1 : -1);
  }
  __syncthreads();
  if (x && c != 0.0)
    for (int e = threadIdx.x; e < 8 * n; e += blockDim.x) xs[e] = x[ro + (size_t)nbr[e / n] * n + e % n];
  __syncthreads();
  const int k = threadIdx.x / n, i = threadIdx.x % n;
  if (k < 8) {
    cplx<T> acc = czero<T>();
    if (x && c != 0.0) {
      const BS* M = blk + (((size_t)site * 9 + 1 + k) * n) * n + i;
      const cplx<T>* xv = xs + k * n;
#pragma unroll 8
      for (int j = 0; j < n; ++j) cfma(acc, ld_cplx(M, (size_t)j * n), xv[j]);
      if (bscale) acc = T(bscale[site]) * acc;
    }
    part[k * n + i] = acc;
  }
  __syncthreads();
  if (threadIdx.x < n) {
    cplx<T> y = czero<T>();
#pragma unroll
    for (int q = 0; q < 8; ++q) y = y + part[q * n + threadIdx.x];
    y = T(c) * y;
    if (b && a != 0.0) y = y + T(a) * b[ro + (size_t)site * n + threadIdx.x];
    u[threadIdx.x] = y;
  }
  __syncthreads();
  if (threadIdx.x < n) {
    cplx<T> acc = czero<T>();
    const cplx<T>* Mi = inv + ((size_t)site * n) * n + threadIdx.x;
#pragma unroll 8
    for (int j = 0; j < n; ++j) cfma(acc, Mi[(size_t)j * n], u[j]);
    t[ro + (size_t)site * n + threadIdx.x] = acc;
  }
}

template <typename T, typename BS>
__global__ void k_schur_even(cplx<T>* __restrict__ y, const cplx<T>* __restrict__ x, const cplx<T>* __restrict__ t,
                             const cplx<T>* __restrict__ b, const BS* __restrict__ blk,
                             const float* __restrict__ bscale, Geom g, int n, size_t rstride, double a, double s,
                             double c) {
  extern __shared__ unsigned char smem_raw[];
  cplx<T>* xs = reinterpret_cast<cplx<T>*>(smem_raw);   // [9][n]
  cplx<T>* part = xs + 9 * n;                           // [9][n]
  __shared__ int nbr[9];
  const int site = blockIdx.x;
  const size_t ro = (size_t)blockIdx.y * rstride;
  int cc[4];
  geom_coords(g, site, cc);
  if (geom_parity(cc) != 0) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) y[ro + (size_t)site * n + i] = czero<T>();
    return;
  }
  if (threadIdx.x < 9) {
    const int k = threadIdx.x;
    nbr[k] = k == 0 ? site : geom_neighbor(g, cc, (k - 1) % 4, k <= 4 ? +1 : -1);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 9 * n; e += blockDim.x) {
    const int k = e / n, j = e % n;
    const cplx<T>* src = k == 0 ? x : t;
    const double w = k == 0 ? s : c;
    xs[e] = (src && w != 0.0) ? src[ro + (size_t)nbr[k] * n + j] : czero<T>();
  }
  __syncthreads();
  const int k = threadIdx.x / n, i = threadIdx.x % n;
  if (k < 9) {
    cplx<T> acc = czero<T>();
    const double w = k == 0 ? s : c;
    if (w != 0.0 && (k == 0 ? x : t)) {
      const BS* M = blk + (((size_t)site * 9 + k) * n) * n + i;
      const cplx<T>* xv = xs + k * n;
#pragma unroll 8
      for (int j = 0; j < n; ++j) cfma(acc, ld_cplx(M, (size_t)j * n), xv[j]);
      if (bscale) acc = T(bscale[site]) * acc;
    }
    part[k * n + i] = T(w) * acc;
  }
  __syncthreads();
  if (threadIdx.x < n) {
    cplx<T> v = czero<T>();
#pragma unroll
    for (int q = 0; q < 9; ++q) v = v + part[q * n + threadIdx.x];
    const size_t o = ro + (size_t)site * n + threadIdx.x;
    if (b && a != 0.0) v = v + T(a) * b[o];
    y[o] = v;
  }
}

// One colour sweep of SAP on a coarse level: one CTA per SAP block; thread t owns
// the rows t, t + blockDim.x, ... (at most RPT) of the block, row = (site, i) in
// block-local order (bsite / bloc tables).  rho = (b - D z)_B, k MR steps on D_B
// (hops leaving the block dropped), z_B += e_B; the operator is read from global
// memory.
template <typename T, typename BS, int RPT>
__global__ void k_coarse_sap(cplx<T>* __restrict__ z, const cplx<T>* __restrict__ bsrc,
                             const BS* __restrict__ blk, const float* __restrict__ bscale, Geom g, int n,
                             size_t rstride, const int* __restrict__ blocks, int k_mr,
                             const int* __restrict__ bsite, const int* __restrict__ bloc) {
  extern __shared__ unsigned char smem_raw[];
  cplx<T>* rs = reinterpret_cast<cplx<T>*>(smem_raw);        // [vB * n]
  T* sh = reinterpret_cast<T*>(rs + (size_t)g.vB * n);          // [warps][3]
  const int b = blocks[blockIdx.x];
  const int rows = g.vB * n;
  const int* bs = bsite + (size_t)b * g.vB;
  const size_t ro = (size_t)blockIdx.y * rstride;
  cplx<T>* pz = z + ro;
  cplx<T> r[RPT], xs[RPT], p[RPT];
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    r[q] = czero<T>();
    xs[q] = czero<T>();
    const int row = threadIdx.x + q * blockDim.x;
    if (row < rows) {
      const int loc = row / n, i = row - loc * n;
      const int site = bs[loc];
      int c[4];
      geom_coords(g, site, c);
      cplx<T> acc = czero<T>();
      // self block, then the forward (1 + mu) and backward (5 + mu) blocks; written as
      // explicit direction loops (a single 9-way loop over k was mis-executed here)
      {
        const cplx<T>* v = pz + (size_t)site * n;
        for (int j = 0; j < n; ++j) cfma(acc, ld_cplx(blk, bidx(site, 0, n, i, j)), v[j]);
      }
      for (int mu = 0; mu < 4; ++mu)
        for (int sd = 0; sd < 2; ++sd) {
          const int dir = sd ? -1 : +1, k = sd ? 5 + mu : 1 + mu;
          const cplx<T>* v = pz + (size_t)geom_neighbor(g, c, mu, dir) * n;
          for (int j = 0; j < n; ++j) cfma(acc, ld_cplx(blk, bidx(site, k, n, i, j)), v[j]);
        }
      const T sc = bscale ? T(bscale[site]) : T(1);
      r[q] = bsrc[ro + (size_t)site * n + i] - sc * acc;
    }
  }
  for (int it = 0; it < k_mr; ++it) {
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      const int row = threadIdx.x + q * blockDim.x;
      if (row < rows) rs[row] = r[q];
    }
    __syncthreads();
    T nre = T(0), nim = T(0), den = T(0);
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      p[q] = czero<T>();
      const int row = threadIdx.x + q * blockDim.x;
      if (row < rows) {
        const int loc = row / n, i = row - loc * n;
        const int site = bs[loc];
        int c[4];
        geom_coords(g, site, c);
        cplx<T> acc = czero<T>();
        {
          const cplx<T>* v = rs + (size_t)loc * n;
#pragma unroll 8
          for (int j = 0; j < n; ++j) cfma(acc, ld_cplx(blk, bidx(site, 0, n, i, j)), v[j]);
        }
        for (int mu = 0; mu < 4; ++mu)
          for (int sd = 0; sd < 2; ++sd) {
            const int dir = sd ? -1 : +1, k = sd ? 5 + mu : 1 + mu;
            if (!hop_internal(g, c, mu, dir, g.B)) continue;
            const cplx<T>* v = rs + (size_t)bloc[geom_neighbor(g, c, mu, dir)] * n;
#pragma unroll 8
            for (int j = 0; j < n; ++j) cfma(acc, ld_cplx(blk, bidx(site, k, n, i, j)), v[j]);
          }
        const T sc = bscale ? T(bscale[site]) : T(1);
        p[q] = sc * acc;
        const cplx<T> tt = cdotc(p[q], r[q]);
        nre += tt.re;
        nim += tt.im;
        den += cnorm2(p[q]);
      }
    }
    cta_sum3(nre, nim, den, sh);
    const cplx<T> alpha = den > T(0) ? cmk<T>(nre / den, nim / den) : czero<T>();
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      cfma(xs[q], alpha, r[q]);
      r[q] = r[q] - alpha * p[q];
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int row = threadIdx.x + q * blockDim.x;
    if (row < rows) {
      const int loc = row / n, i = row - loc * n;
      const size_t a = ro + (size_t)bs[loc] * n + i;
      z[a] = z[a] + xs[q];
    }
  }
}

// shared-memory layout of k_coarse_sap_cluster (byte offsets, 16-byte aligned)
struct SapSmem {
  size_t rfull, pbuf, part, red, sh, slot, bar, total;
};
DD_HD size_t al16(size_t x) { return (x + 15) & ~size_t(15); }
DD_HD SapSmem sap_smem_layout(int vB, int n, int spc, int nsl, size_t bs, size_t ts) {
  SapSmem L;
  size_t o = al16((size_t)spc * nsl * n * n * bs);
  L.rfull = o;
  o = al16(o + (size_t)vB * n * 2 * ts);
  L.pbuf = o;
  o = al16(o + (size_t)2 * vB * n * 2 * ts);
  L.part = o;
  o = al16(o + (size_t)9 * spc * n * 2 * ts);
  L.red = o;
  o = al16(o + (size_t)2 * 16 * 4 * ts);
  L.sh = o;
  o = al16(o + (size_t)(32 * 3 + 4) * ts);
  L.slot = o;
  o = al16(o + (size_t)spc * 9 * sizeof(int));
  L.bar = o;
  L.total = al16(o + 8);
  return L;
}

// SAP colour sweep on a coarse level with one thread-block cluster per SAP
// block.  CTA q of the cluster owns `spc` sites of the block, one thread per
// (row, block k) of its sites.  The blocks of its sites that couple inside the
// SAP block (self block included) are staged once into shared memory by bulk
// copies; the hops leaving the block are only needed for rho = b - D z and are
// read from global memory.  Every CTA keeps the whole block residual r and the
// whole MR direction p = D_B r in shared memory: after computing p on its own
// rows a CTA writes them, with its partial dot products, into every CTA of the
// cluster (distributed shared memory), so each MR step needs one cluster
// barrier; p and the partials are double-buffered across steps.  The partial
// dot products are summed in rank order, so every CTA computes the same alpha
// and applies r <- r - alpha p to its whole copy.  Same arithmetic as
// k_coarse_sap: rho = (b - D z)_B, k MR steps on D_B, z_B += e_B.
template <typename T, typename BS>
__global__ void __launch_bounds__(768, 2) k_coarse_sap_cluster(cplx<T>* __restrict__ z, const cplx<T>* __restrict__ bsrc,
                                     const BS* __restrict__ blk, const float* __restrict__ bscale, Geom g, int n,
                                     size_t rstride, int nrhs, const int* __restrict__ blocks, int k_mr, int spc,
                                     int nsl, int* err, const int* __restrict__ bsite,
                                     const int* __restrict__ bloc) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // the next sweep (launched with programmatic stream serialization) may stage its blocks while
  // this one runs; it waits for this grid before reading z or b
  pdl_launch_dependents();
  cg::cluster_group cluster = cg::this_cluster();
  const int CLS = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int vB = g.vB;
  const int b = blocks[blockIdx.x / CLS];
  const int rows = spc * n;
  const size_t nn = (size_t)n * n;
  const SapSmem L = sap_smem_layout(vB, n, spc, nsl, sizeof(BS), sizeof(T));
  BS* stage = reinterpret_cast<BS*>(smem_raw);                                // [spc][nsl][n][n]
  cplx<T>* rfull = reinterpret_cast<cplx<T>*>(smem_raw + L.rfull);            // [vB*n]
  cplx<T>* pbuf = reinterpret_cast<cplx<T>*>(smem_raw + L.pbuf);              // [2][vB*n]
  cplx<T>* part = reinterpret_cast<cplx<T>*>(smem_raw + L.part);              // [9][rows]
  T* red = reinterpret_cast<T*>(smem_raw + L.red);                            // [2][16][4]
  T* sh = reinterpret_cast<T*>(smem_raw + L.sh);                              // [32][3] + 3
  int* slot = reinterpret_cast<int*>(smem_raw + L.slot);                      // [spc][9]
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem_raw + L.bar);
  const int* own = bsite + (size_t)b * vB + rank * spc;   // own sites, block-local order
  // slot of block k of own site sl in the staged array (-1: the hop leaves the SAP block)
  if (threadIdx.x < spc) {
    int c[4];
    geom_coords(g, own[threadIdx.x], c);
    // slots in k order (self, forward mu = 0..3, backward mu = 0..3), explicit direction loops
    int* sl9 = slot + threadIdx.x * 9;
    int ns = 0;
    sl9[0] = ns++;
    for (int sd = 0; sd < 2; ++sd)
      for (int mu = 0; mu < 4; ++mu)
        sl9[(sd ? 5 : 1) + mu] = hop_internal(g, c, mu, sd ? -1 : +1, g.B) ? ns++ : -1;
  }
  if (threadIdx.x == 0) mbar_init(bar, 1);
  __syncthreads();
  if (threadIdx.x < 32) {
    int cnt = 0;
    for (int e = 0; e < spc * 9; ++e) cnt += slot[e] >= 0 ? 1 : 0;
    if (threadIdx.x == 0) mbar_arrive_expect_tx(bar, (unsigned)(cnt * nn * sizeof(BS)));
    __syncwarp();
    for (int e = threadIdx.x; e < spc * 9; e += 32) {
      const int sl = e / 9, k = e % 9, q = slot[e];
      if (q >= 0)
        bulk_g2s(stage + ((size_t)sl * nsl + q) * nn, blk + ((size_t)own[sl] * 9 + k) * nn,
                 (unsigned)(nn * sizeof(BS)), bar);
    }
  }
  const int k = threadIdx.x / rows;
  const int rl = threadIdx.x - k * rows;
  const int sl = rl / n, i = rl - (rl / n) * n;
  const int site = own[sl];
  const T sc = bscale ? T(bscale[site]) : T(1);
  int q = -1, nb = site, nloc = 0;
  if (k < 9) {
    q = slot[sl * 9 + k];
    if (k > 0) {
      int c[4];
      geom_coords(g, site, c);
      nb = geom_neighbor(g, c, (k - 1) % 4, k <= 4 ? +1 : -1);
    }
    nloc = q >= 0 ? bloc[nb] : 0;
  }
  const BS* Ms = stage + ((size_t)sl * nsl + (q >= 0 ? q : 0)) * nn + i;   // staged row i (column-major)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  int ok = 1;
  pdl_wait();   // the previous kernel's z and b are complete from here on
  // the right-hand sides of the batch one after the other, on the blocks staged once
  for (int rh = 0; rh < nrhs; ++rh) {
    const size_t ro = (size_t)rh * rstride;
    // rho = b - D z on the own rows: hops leaving the block from global memory ...
    cplx<T> acc = czero<T>();
    if (k < 9 && q < 0) {
      const BS* M = blk + ((size_t)site * 9 + k) * nn + i;
      const cplx<T>* v = z + ro + (size_t)nb * n;
#pragma unroll 8
      for (int j = 0; j < n; ++j) cfma(acc, ld_cplx(M, (size_t)j * n), v[j]);
    }
    if (rh == 0) {
      ok = __syncthreads_and(mbar_wait_bounded(bar, 0) ? 1 : 0);
      if (!ok && threadIdx.x == 0) atomicExch(err, 2);
    }
    // ... and the blocks inside it from shared memory
    if (k < 9 && q >= 0) {
      const cplx<T>* v = z + ro + (size_t)nb * n;
#pragma unroll 8
      for (int j = 0; j < n; ++j) cfma(acc, ld_cplx(Ms, (size_t)j * n), v[j]);
    }
    if (k < 9) part[k * rows + rl] = sc * acc;
    __syncthreads();
    cplx<T> r = czero<T>(), xs = czero<T>();
    if (threadIdx.x < rows) {
      cplx<T> d = czero<T>();
#pragma unroll
      for (int m = 0; m < 9; ++m) d = d + part[m * rows + threadIdx.x];
      r = bsrc[ro + (size_t)own[threadIdx.x / n] * n + threadIdx.x % n] - d;
      for (int c = 0; c < CLS; ++c) cluster.map_shared_rank(rfull, c)[(size_t)rank * rows + threadIdx.x] = r;
    }
    cluster.sync();
    for (int it = 0; it < k_mr; ++it) {
      const int buf = it & 1;
      cplx<T>* pb = pbuf + (size_t)buf * vB * n;
      T* rb = red + buf * 64;
      // p = D_B r on the own rows, from the staged blocks and the local copy of r
      if (k < 9) {
        cplx<T> a = czero<T>();
        if (q >= 0) {
          const cplx<T>* v = rfull + (size_t)nloc * n;
#pragma unroll 8
          for (int j = 0; j < n; ++j) cfma(a, ld_cplx(Ms, (size_t)j * n), v[j]);
        }
        part[k * rows + rl] = sc * a;
      }
      __syncthreads();
      cplx<T> p = czero<T>();
      T nre = T(0), nim = T(0), den = T(0);
      if (threadIdx.x < rows) {
#pragma unroll
        for (int m = 0; m < 9; ++m) p = p + part[m * rows + threadIdx.x];
        const cplx<T> t = cdotc(p, r);
        nre = t.re;
        nim = t.im;
        den = cnorm2(p);
        for (int c = 0; c < CLS; ++c) cluster.map_shared_rank(pb, c)[(size_t)rank * rows + threadIdx.x] = p;
      }
      for (int off = 16; off >= 1; off >>= 1) {
        nre += __shfl_xor_sync(0xffffffffu, nre, off);
        nim += __shfl_xor_sync(0xffffffffu, nim, off);
        den += __shfl_xor_sync(0xffffffffu, den, off);
      }
      if (lane == 0) { sh[3 * warp] = nre; sh[3 * warp + 1] = nim; sh[3 * warp + 2] = den; }
      __syncthreads();
      if (warp == 0) {   // warp partials summed by a shuffle tree (fixed order), then sent to every CTA
        T a = lane < nw ? sh[3 * lane] : T(0);
        T bb = lane < nw ? sh[3 * lane + 1] : T(0);
        T cc = lane < nw ? sh[3 * lane + 2] : T(0);
        for (int off = 16; off >= 1; off >>= 1) {
          a += __shfl_xor_sync(0xffffffffu, a, off);
          bb += __shfl_xor_sync(0xffffffffu, bb, off);
          cc += __shfl_xor_sync(0xffffffffu, cc, off);
        }
        if (lane < CLS) {
          T* dst = cluster.map_shared_rank(rb, lane) + rank * 4;
          dst[0] = a;
          dst[1] = bb;
          dst[2] = cc;
        }
      }
      cluster.sync();
      T a = T(0), bb = T(0), cc = T(0);
      for (int c = 0; c < CLS; ++c) { a += rb[c * 4]; bb += rb[c * 4 + 1]; cc += rb[c * 4 + 2]; }
      const cplx<T> alpha = cc > T(0) ? cmk<T>(a / cc, bb / cc) : czero<T>();
      if (threadIdx.x < rows) {
        cfma(xs, alpha, r);
        r = r - alpha * p;
      }
      for (int e = threadIdx.x; e < vB * n; e += blockDim.x) rfull[e] = rfull[e] - alpha * pb[e];
      __syncthreads();
    }
    if (ok && threadIdx.x < rows) {
      const size_t a = ro + (size_t)own[threadIdx.x / n] * n + threadIdx.x % n;
      z[a] = z[a] + xs;
    }
    // every CTA is done with its copies of r, p and the partials before the next right-hand side
    // writes into them
    if (rh + 1 < nrhs) cluster.sync();
  }
  if (!ok && threadIdx.x == 0) mbar_wait_bounded(bar, 0);   // no copy may still be in flight at exit
}

// ---------------------------------------------------------------------------
// Persistent coarse SAP: all `iters` SAP applications (a red then a black sweep each) of one
// smoother call in one launch, for levels whose SAP blocks of both colours are resident at once.
// Cluster c owns red block blocks0[c] and black block blocks1[c]; each CTA stages the blocks
// inside both SAP blocks of its sites once, for the whole call.  A colour sweep is the sweep of
// k_coarse_sap_cluster (same arithmetic, same order); sweeps are separated by a barrier over all
// clusters, which the cooperative launch makes safe (all CTAs co-resident).  z is read through
// L2 (ld.global.cg): values written by other SMs in the previous sweep are never taken from a
// stale L1 line.

// z in L2 only (values written by other CTAs of the launch)
__device__ __forceinline__ cplx<float> ldz(const cplx<float>* p) {
  const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
  return cmk<float>(v.x, v.y);
}
__device__ __forceinline__ cplx<double> ldz(const cplx<double>* p) {
  const double2 v = __ldcg(reinterpret_cast<const double2*>(p));
  return cmk<double>(v.x, v.y);
}

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Barrier over the clusters of a persistent launch.  Rank 0 of every cluster counts its cluster
// in (the counter is zeroed before the launch; round r is complete at ncl * (r + 1)) and waits
// for the others; the wait is bounded (about a second at the maximum clock), after which
// *err = 3 and every CTA of the cluster gets false.
__device__ bool persist_grid_sync(unsigned* cnt, unsigned target, cg::cluster_group& cluster, int* flag, int* err) {
  cluster.sync();   // the sweep's writes of every CTA of the cluster precede the arrival
  if (cluster.block_rank() == 0 && threadIdx.x == 0) {
    __threadfence();
    atomicAdd(cnt, 1u);
    const long long t0 = clock64();
    int ok = 1;
    while (ld_acquire_gpu(cnt) < target) {
      if (clock64() - t0 > 2000000000LL) {
        ok = 0;
        atomicExch(err, 3);
        break;
      }
      __nanosleep(64);
    }
    *flag = ok;
  }
  cluster.sync();
  return *cluster.map_shared_rank(flag, 0) != 0;
}

struct PSapSmem {
  size_t rfull, pbuf, part, red, sh, slot, flag, bar, total;
};
// nbpc SAP blocks of each colour per cluster; rows = nbpc * spc * n per CTA
DD_HD PSapSmem psap_smem_layout(int vB, int n, int spc, int nsl, int nbpc, size_t bs, size_t ts) {
  PSapSmem L;
  size_t o = al16((size_t)2 * nbpc * spc * nsl * n * n * bs);
  L.rfull = o;
  o = al16(o + (size_t)nbpc * vB * n * 2 * ts);
  L.pbuf = o;
  o = al16(o + (size_t)2 * nbpc * vB * n * 2 * ts);
  L.part = o;
  o = al16(o + (size_t)9 * nbpc * spc * n * 2 * ts);
  L.red = o;
  o = al16(o + (size_t)2 * nbpc * 16 * 4 * ts);
  L.sh = o;
  o = al16(o + (size_t)(32 * 3 * nbpc + 4) * ts);
  L.slot = o;
  o = al16(o + (size_t)2 * nbpc * spc * 9 * sizeof(int));
  L.flag = o;
  o = al16(o + 16);
  L.bar = o;
  L.total = al16(o + 8);
  return L;
}

// NB SAP blocks of each colour per cluster (1 or 2): CTA rank q owns sites q*spc .. q*spc+spc-1
// of each of them; the rows of block j are rows j*spc*n .. (j+1)*spc*n-1 of the CTA, with their
// own residual copy, MR direction and dot products.
template <typename T, typename BS, int NB>
__global__ void __launch_bounds__(768, 1) k_coarse_sap_persist(
    cplx<T>* __restrict__ z, const cplx<T>* __restrict__ bsrc, const BS* __restrict__ blk,
    const float* __restrict__ bscale, Geom g, int n, size_t rstride, int nrhs, const int* __restrict__ blocks0,
    int nb0, const int* __restrict__ blocks1, int nb1, int k_mr, int spc, int nsl, int iters, int* err,
    const int* __restrict__ bsite, const int* __restrict__ bloc, unsigned* gcnt) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  cg::cluster_group cluster = cg::this_cluster();
  const int CLS = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int cid = blockIdx.x / CLS;
  const unsigned ncl = gridDim.x / CLS;
  const int vB = g.vB;
  const int rb = spc * n;          // rows of one block in this CTA
  const int rows = NB * rb;
  const size_t nn = (size_t)n * n;
  const PSapSmem L = psap_smem_layout(vB, n, spc, nsl, NB, sizeof(BS), sizeof(T));
  BS* stage = reinterpret_cast<BS*>(smem_raw);                                // [2][NB*spc][nsl][n][n]
  cplx<T>* rfull = reinterpret_cast<cplx<T>*>(smem_raw + L.rfull);            // [NB][vB*n]
  cplx<T>* pbuf = reinterpret_cast<cplx<T>*>(smem_raw + L.pbuf);              // [2][NB][vB*n]
  cplx<T>* part = reinterpret_cast<cplx<T>*>(smem_raw + L.part);              // [9][rows]
  T* red = reinterpret_cast<T*>(smem_raw + L.red);                            // [2][NB][16][4]
  T* sh = reinterpret_cast<T*>(smem_raw + L.sh);                              // [32][3*NB] + 4
  int* slot = reinterpret_cast<int*>(smem_raw + L.slot);                      // [2][NB*spc][9]
  int* flag = reinterpret_cast<int*>(smem_raw + L.flag);
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem_raw + L.bar);
  // block of colour c, slot j of this cluster (-1: none)
  auto block_of = [&](int c, int j) -> int {
    const int q = cid * NB + j;
    return c ? (q < nb1 ? blocks1[q] : -1) : (q < nb0 ? blocks0[q] : -1);
  };
  // slots of the staged blocks (k order: self, forward mu, backward mu)
  if (threadIdx.x < 2 * NB * spc) {
    const int c = threadIdx.x / (NB * spc), js = threadIdx.x - c * NB * spc;
    const int j = js / spc, s = js - j * spc;
    int* sl9 = slot + (c * NB * spc + js) * 9;
    const int bc = block_of(c, j);
    if (bc >= 0) {
      int co[4];
      geom_coords(g, bsite[(size_t)bc * vB + rank * spc + s], co);
      int ns = 0;
      sl9[0] = ns++;
      for (int sd = 0; sd < 2; ++sd)
        for (int mu = 0; mu < 4; ++mu)
          sl9[(sd ? 5 : 1) + mu] = hop_internal(g, co, mu, sd ? -1 : +1, g.B) ? ns++ : -1;
    } else {
      for (int e = 0; e < 9; ++e) sl9[e] = -1;
    }
  }
  if (threadIdx.x == 0) mbar_init(bar, 1);
  __syncthreads();
  if (threadIdx.x < 32) {
    int cnt = 0;
    for (int e = 0; e < 2 * NB * spc * 9; ++e) cnt += slot[e] >= 0 ? 1 : 0;
    if (threadIdx.x == 0) mbar_arrive_expect_tx(bar, (unsigned)(cnt * nn * sizeof(BS)));
    __syncwarp();
    for (int e = threadIdx.x; e < 2 * NB * spc * 9; e += 32) {
      const int cjs = e / 9, k = e % 9, q = slot[e];   // cjs = (c * NB + j) * spc + s
      if (q >= 0) {
        const int c = cjs / (NB * spc), js = cjs - c * NB * spc;
        const int j = js / spc, s = js - j * spc;
        const int site = bsite[(size_t)block_of(c, j) * vB + rank * spc + s];
        bulk_g2s(stage + ((size_t)cjs * nsl + q) * nn, blk + ((size_t)site * 9 + k) * nn,
                 (unsigned)(nn * sizeof(BS)), bar);
      }
    }
  }
  const int ok = __syncthreads_and(mbar_wait_bounded(bar, 0) ? 1 : 0);
  if (!ok && threadIdx.x == 0) atomicExch(err, 2);
  const int k = threadIdx.x / rows;
  const int rl = threadIdx.x - k * rows;
  const int jb = rl / rb, rj = rl - jb * rb;      // block of the row, row inside that block's share
  const int sl = rj / n, i = rj - (rj / n) * n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  // the rows this thread owns as a residual row (threadIdx.x < rows): block jr, local row rr
  const int jr = threadIdx.x / rb, rr = threadIdx.x - (threadIdx.x / rb) * rb;
  unsigned round = 0;
  bool alive = true;
  for (int it = 0; it < iters && alive; ++it)
    for (int c = 0; c < 2 && alive; ++c) {
      const int bk = k < 9 ? block_of(c, jb) : -1;            // this thread's (row, k) block
      const int bres = threadIdx.x < rows ? block_of(c, jr) : -1;   // this thread's residual row's block
      const bool any = block_of(c, 0) >= 0;                    // uniform over the cluster
      if (any) {
        int site = 0, q = -1, nb = 0, nloc = 0;
        T sc = T(1);
        if (bk >= 0) {
          site = bsite[(size_t)bk * vB + rank * spc + sl];
          sc = bscale ? T(bscale[site]) : T(1);
          nb = site;
          q = slot[((c * NB + jb) * spc + sl) * 9 + k];
          if (k > 0) {
            int co[4];
            geom_coords(g, site, co);
            nb = geom_neighbor(g, co, (k - 1) % 4, k <= 4 ? +1 : -1);
          }
          nloc = q >= 0 ? bloc[nb] : 0;
        }
        const BS* Ms = stage + ((size_t)((c * NB + jb) * spc + sl) * nsl + (q >= 0 ? q : 0)) * nn + i;
        const int* ownr = bres >= 0 ? bsite + (size_t)bres * vB + rank * spc : nullptr;
        for (int rh = 0; rh < nrhs; ++rh) {
          const size_t ro = (size_t)rh * rstride;
          // rho = b - D z on the own rows (z through L2)
          if (k < 9) {
            cplx<T> acc = czero<T>();
            if (bk >= 0) {
              const cplx<T>* v = z + ro + (size_t)nb * n;
              if (q < 0) {
                const BS* M = blk + ((size_t)site * 9 + k) * nn + i;
#pragma unroll 8
                for (int j = 0; j < n; ++j) cfma(acc, ld_cplx(M, (size_t)j * n), ldz(v + j));
              } else {
#pragma unroll 8
                for (int j = 0; j < n; ++j) cfma(acc, ld_cplx(Ms, (size_t)j * n), ldz(v + j));
              }
            }
            part[k * rows + rl] = sc * acc;
          }
          __syncthreads();
          cplx<T> r = czero<T>(), xs = czero<T>();
          if (bres >= 0) {
            cplx<T> d = czero<T>();
#pragma unroll
            for (int m = 0; m < 9; ++m) d = d + part[m * rows + threadIdx.x];
            r = bsrc[ro + (size_t)ownr[rr / n] * n + rr % n] - d;
            for (int cc = 0; cc < CLS; ++cc)
              cluster.map_shared_rank(rfull + (size_t)jr * vB * n, cc)[(size_t)rank * rb + rr] = r;
          }
          cluster.sync();
          for (int mr = 0; mr < k_mr; ++mr) {
            const int buf = mr & 1;
            cplx<T>* pb = pbuf + (size_t)buf * NB * vB * n;
            T* rbf = red + buf * NB * 64;
            // p = D_B r on the own rows, from the staged blocks and the local copy of r
            if (k < 9) {
              cplx<T> a = czero<T>();
              if (bk >= 0 && q >= 0) {
                const cplx<T>* v = rfull + (size_t)jb * vB * n + (size_t)nloc * n;
#pragma unroll 8
                for (int j = 0; j < n; ++j) cfma(a, ld_cplx(Ms, (size_t)j * n), v[j]);
              }
              part[k * rows + rl] = sc * a;
            }
            __syncthreads();
            cplx<T> p = czero<T>();
            T v3[3 * NB];
#pragma unroll
            for (int e = 0; e < 3 * NB; ++e) v3[e] = T(0);
            if (bres >= 0) {
#pragma unroll
              for (int m = 0; m < 9; ++m) p = p + part[m * rows + threadIdx.x];
              const cplx<T> t = cdotc(p, r);
#pragma unroll
              for (int jj = 0; jj < NB; ++jj)
                if (jj == jr) {
                  v3[3 * jj] = t.re;
                  v3[3 * jj + 1] = t.im;
                  v3[3 * jj + 2] = cnorm2(p);
                }
              for (int cc = 0; cc < CLS; ++cc)
                cluster.map_shared_rank(pb + (size_t)jr * vB * n, cc)[(size_t)rank * rb + rr] = p;
            }
#pragma unroll
            for (int e = 0; e < 3 * NB; ++e)
              for (int off = 16; off >= 1; off >>= 1) v3[e] += __shfl_xor_sync(0xffffffffu, v3[e], off);
            if (lane == 0)
#pragma unroll
              for (int e = 0; e < 3 * NB; ++e) sh[3 * NB * warp + e] = v3[e];
            __syncthreads();
            if (warp == 0) {   // warp partials summed by a shuffle tree (fixed order), sent to every CTA
#pragma unroll
              for (int e = 0; e < 3 * NB; ++e) {
                T a = lane < nw ? sh[3 * NB * lane + e] : T(0);
                for (int off = 16; off >= 1; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
                v3[e] = a;
              }
              if (lane < CLS)
#pragma unroll
                for (int jj = 0; jj < NB; ++jj) {
                  T* dst = cluster.map_shared_rank(rbf + jj * 64, lane) + rank * 4;
                  dst[0] = v3[3 * jj];
                  dst[1] = v3[3 * jj + 1];
                  dst[2] = v3[3 * jj + 2];
                }
            }
            cluster.sync();
            cplx<T> alpha[NB];
#pragma unroll
            for (int jj = 0; jj < NB; ++jj) {
              T a = T(0), bb = T(0), cc = T(0);
              for (int q2 = 0; q2 < CLS; ++q2) {
                a += rbf[jj * 64 + q2 * 4];
                bb += rbf[jj * 64 + q2 * 4 + 1];
                cc += rbf[jj * 64 + q2 * 4 + 2];
              }
              alpha[jj] = cc > T(0) ? cmk<T>(a / cc, bb / cc) : czero<T>();
            }
            if (bres >= 0) {
              cplx<T> al = alpha[0];
#pragma unroll
              for (int jj = 1; jj < NB; ++jj)
                if (jj == jr) al = alpha[jj];
              cfma(xs, al, r);
              r = r - al * p;
            }
            for (int e = threadIdx.x; e < NB * vB * n; e += blockDim.x) {
              const int jj = e / (vB * n);
              cplx<T> al = alpha[0];
#pragma unroll
              for (int j2 = 1; j2 < NB; ++j2)
                if (j2 == jj) al = alpha[j2];
              rfull[e] = rfull[e] - al * pb[e];
            }
            __syncthreads();
          }
          if (ok && bres >= 0) {
            const size_t a = ro + (size_t)ownr[rr / n] * n + rr % n;
            z[a] = ldz(z + a) + xs;
          }
          // every CTA is done with its copies of r, p and the partials before the next right-hand
          // side writes into them
          if (rh + 1 < nrhs) cluster.sync();
        }
      }
      if (it + 1 < iters || c == 0) {
        ++round;
        alive = persist_grid_sync(gcnt, ncl * round, cluster, flag, err);
      }
    }
  if (!ok && threadIdx.x == 0) mbar_wait_bounded(bar, 0);   // no copy may still be in flight at exit
  cluster.sync();   // no CTA exits while others may still write into its shared memory
}

// Gauss-Jordan inversion with partial pivoting of every self block (FP64).
__global__ void k_selfinv_build(cplx<double>* __restrict__ inv, const cplx<double>* __restrict__ blk, int n,
                                int* err) {
  extern __shared__ unsigned char smem_raw[];
  cplx<double>* a = reinterpret_cast<cplx<double>*>(smem_raw);   // [n][2n] row-major
  cplx<double>* fac = a + (size_t)n * 2 * n;                       // [n] column k before elimination
  __shared__ int piv;
  const int site = blockIdx.x;
  const int w = 2 * n;
  for (int e = threadIdx.x; e < n * w; e += blockDim.x) {
    const int i = e / w, j = e % w;
    a[e] = j < n ? blk[bidx(site, 0, n, i, j)] : cmk(i == j - n ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x == 0) {
      int p = k;
      double best = cnorm2(a[k * w + k]);
      for (int i = k + 1; i < n; ++i) {
        const double v = cnorm2(a[i * w + k]);
        if (v > best) { best = v; p = i; }
      }
      piv = best > 0.0 ? p : -1;
    }
    __syncthreads();
    if (piv < 0) {
      if (threadIdx.x == 0) atomicExch(err, 1);
      return;
    }
    if (piv != k)
      for (int j = threadIdx.x; j < w; j += blockDim.x) {
        const cplx<double> t = a[k * w + j];
        a[k * w + j] = a[piv * w + j];
        a[piv * w + j] = t;
      }
    __syncthreads();
    const cplx<double> d = a[k * w + k];
    const double dn = cnorm2(d);
    const cplx<double> dinv = cmk(d.re / dn, -d.im / dn);
    __syncthreads();
    for (int j = threadIdx.x; j < w; j += blockDim.x) a[k * w + j] = a[k * w + j] * dinv;
    for (int i = threadIdx.x; i < n; i += blockDim.x) fac[i] = a[i * w + k];
    __syncthreads();
    for (int e = threadIdx.x; e < n * w; e += blockDim.x) {
      const int i = e / w, j = e % w;
      if (i != k) a[e] = a[e] - fac[i] * a[k * w + j];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e % n, j = e / n;
    inv[((size_t)site * n + j) * n + i] = a[i * w + n + j];
  }
}

template <typename T>
__global__ void k_selfinv_apply(cplx<T>* __restrict__ out, const cplx<T>* __restrict__ in,
                                const cplx<T>* __restrict__ inv, Geom g, int n, int parity, size_t rstride) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)g.V * n) return;
  const int site = (int)(t / n), i = (int)(t % n);
  const size_t ro = (size_t)blockIdx.y * rstride;
  int c[4];
  geom_coords(g, site, c);
  cplx<T> acc = czero<T>();
  if (parity < 0 || geom_parity(c) == parity) {
    const cplx<T>* v = in + ro + (size_t)site * n;
    for (int j = 0; j < n; ++j) cfma(acc, inv[((size_t)site * n + j) * n + i], v[j]);
  }
  out[ro + t] = acc;
}

template <typename T>
__global__ void k_sub_parity(cplx<T>* y, const cplx<T>* a, const cplx<T>* b,
                             Geom g, int n, int parity, size_t rstride) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)g.V * n) return;
  const int site = (int)(t / n);
  const size_t ro = (size_t)blockIdx.y * rstride;
  int c[4];
  geom_coords(g, site, c);
  const bool keep = parity < 0 || geom_parity(c) == parity;
  y[ro + t] = keep ? a[ro + t] - (b ? b[ro + t] : czero<T>()) : czero<T>();
}

template <typename T>
__global__ void k_coarse_import(cplx<T>* __restrict__ dst, const cplx<double>* __restrict__ src, Geom g, int n,
                                size_t rstride) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)g.V * n) return;
  const int site = (int)(t / n), i = (int)(t % n);
  int c[4];
  geom_coords(g, site, c);
  const size_t lex = (size_t)lin4(c, g.L);
  dst[(size_t)blockIdx.y * rstride + t] = ccast<T>(src[(size_t)blockIdx.y * g.V * n + lex * n + i]);
}

template <typename T>
__global__ void k_coarse_export(cplx<double>* __restrict__ dst, const cplx<T>* __restrict__ src, Geom g, int n,
                                size_t rstride) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)g.V * n) return;
  const int site = (int)(t / n), i = (int)(t % n);
  int c[4];
  geom_coords(g, site, c);
  const size_t lex = (size_t)lin4(c, g.L);
  dst[(size_t)blockIdx.y * g.V * n + lex * n + i] = ccast<double>(src[(size_t)blockIdx.y * rstride + t]);
}

// internal [V][9][n][n] column-major  ->  ABI [lex][9][n][n] row-major
__global__ void k_blocks_export(cplx<double>* __restrict__ dst, const cplx<double>* __restrict__ blk, Geom g, int n) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t per = (size_t)9 * n * n;
  if (t >= (size_t)g.V * per) return;
  const int site = (int)(t / per);
  const size_t r = t % per;
  const int k = (int)(r / ((size_t)n * n));
  const int e = (int)(r % ((size_t)n * n));
  const int i = e / n, j = e % n;
  int c[4];
  geom_coords(g, site, c);
  const size_t lex = (size_t)lin4(c, g.L);
  dst[lex * per + (size_t)k * n * n + (size_t)i * n + j] = blk[bidx(site, k, n, i, j)];
}

// FP16 copy of one site's 9 blocks: s = float(max |re|, |im|), q = RNE_half(x / s)
__global__ void k_blocks_to_half(__half2* __restrict__ dst, float* __restrict__ scale,
                                 const cplx<double>* __restrict__ blk, int n) {
  __shared__ double sh[32];
  const size_t per = (size_t)9 * n * n;
  const cplx<double>* src = blk + (size_t)blockIdx.x * per;
  double mx = 0.0;
  for (size_t e = threadIdx.x; e < per; e += blockDim.x) mx = fmax(mx, fmax(fabs(src[e].re), fabs(src[e].im)));
  for (int off = 16; off >= 1; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, sh[w]);
    const float sf = m > 0.0 ? (float)m : 1.0f;
    scale[blockIdx.x] = sf;
    sh[0] = (double)sf;
  }
  __syncthreads();
  const double sc = sh[0];
  __half2* d = dst + (size_t)blockIdx.x * per;
  for (size_t e = threadIdx.x; e < per; e += blockDim.x)
    d[e] = __halves2half2(__double2half(src[e].re / sc), __double2half(src[e].im / sc));
}

}  // namespace

namespace dd {

void blocks_to_half(__half2* dst, float* scale, const cplx<double>* blk, int V, int n, cudaStream_t st) {
  count_launch();
  k_blocks_to_half<<<V, 256, 0, st>>>(dst, scale, blk, n);
}

template <typename T>
void coarse_apply(cplx<T>* out, const cplx<T>* in, const cplx<T>* b, const CoarseOp<T>& op, int nrhs, size_t rstride,
                  int sel, int sel_mu, int in_chir, cudaStream_t st) {
  const int threads = ((9 * op.n + 31) / 32) * 32;
  const size_t sm = (size_t)18 * op.n * sizeof(cplx<T>);
  dim3 grid(op.g.V, nrhs);
  if constexpr (sizeof(T) == 4) {
    // the whole operator on FP16 storage: the tensor-core kernel where the autotuner chose it
    if (op.blkh && op.tc_ks > 0 && sel == SEL_FULL && in_chir < 0) {
      if (coarse_apply_tc(out, in, b, op, nrhs, rstride, op.tc_ks, st) == cudaSuccess) return;
      cudaGetLastError();
    }
  }
  count_launch();
  if constexpr (sizeof(T) == 4) {
    if (op.blkh) {
      if (b)
        k_coarse_apply<float, true, __half2><<<grid, threads, sm, st>>>(out, in, b, op.blkh, op.bscale, op.g, op.n,
                                                                         rstride, sel, sel_mu, in_chir);
      else
        k_coarse_apply<float, false, __half2><<<grid, threads, sm, st>>>(out, in, b, op.blkh, op.bscale, op.g, op.n,
                                                                          rstride, sel, sel_mu, in_chir);
      return;
    }
  }
  if (b)
    k_coarse_apply<T, true, cplx<T>><<<grid, threads, sm, st>>>(out, in, b, op.blk, nullptr, op.g, op.n, rstride, sel,
                                                                 sel_mu, in_chir);
  else
    k_coarse_apply<T, false, cplx<T>><<<grid, threads, sm, st>>>(out, in, b, op.blk, nullptr, op.g, op.n, rstride,
                                                                  sel, sel_mu, in_chir);
}

// staged blocks per site of the cluster SAP: the self block plus the hops that stay inside
// the SAP block, maximised over the sites of a block (every block has the same shape)
int coarse_sap_slots(const Geom& g) {
  int best = 1;
  for (int loc = 0; loc < g.vB; ++loc) {
    int c[4];
    delin4(loc, g.B, c);   // the sites of the block at the origin
    int cnt = 1;
    for (int k = 1; k < 9; ++k) cnt += hop_internal(g, c, (k - 1) % 4, k <= 4 ? +1 : -1, g.B) ? 1 : 0;
    best = cnt > best ? cnt : best;
  }
  return best;
}

// The dynamic shared-memory limit of a kernel is a process-wide attribute: it is raised to the
// device maximum (not to this plan's size), so that a hierarchy set up later with smaller blocks
// cannot lower it below what an earlier hierarchy's launches use.
template <typename T, typename BS>
void sap_cluster_attrs(size_t smem, int CLS) {
  if (cudaFuncSetAttribute(k_coarse_sap_cluster<T, BS>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024) !=
      cudaSuccess) {
    cudaGetLastError();
    cudaFuncSetAttribute(k_coarse_sap_cluster<T, BS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  }
  if (CLS > 8) cudaFuncSetAttribute(k_coarse_sap_cluster<T, BS>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

// cluster plan of the coarse SAP: cluster size CLS, sites per CTA and staged blocks per
// site (0 if no plan fits).  Sized for operator storage in the compute precision, which
// also covers the FP16 storage.
template <typename T>
int coarse_sap_cluster_plan(const Geom& g, int n, int* CLS_out, int* spc_out, int* nsl_out, int prefer) {
  const int nsl = coarse_sap_slots(g);
  for (int CLS : {prefer, 16, 8, 4, 2}) {
    if (CLS != 2 && CLS != 4 && CLS != 8 && CLS != 16) continue;
    if (g.vB % CLS) continue;
    const int spc = g.vB / CLS;
    const int threads = ((9 * spc * n + 31) / 32) * 32;
    if (threads > 768) continue;   // launch bounds of k_coarse_sap_cluster
    const size_t sm = sap_smem_layout(g.vB, n, spc, nsl, sizeof(cplx<T>), sizeof(T)).total;
    if (sm > 227 * 1024) continue;
    sap_cluster_attrs<T, cplx<T>>(sm, CLS);
    if constexpr (sizeof(T) == 4) sap_cluster_attrs<float, __half2>(sm, CLS);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CLS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(CLS, 1, 1);
    cfg.blockDim = dim3(threads, 1, 1);
    cfg.dynamicSmemBytes = sm;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, k_coarse_sap_cluster<T, cplx<T>>, &cfg) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (nclusters < 1) continue;
    *CLS_out = CLS;
    *spc_out = spc;
    *nsl_out = nsl;
    return 1;
  }
  return 0;
}

// Persistent SAP on FP16 blocks (FP32 compute): the launch's shared memory and threads for nbpc
// SAP blocks of each colour per cluster, and whether all clusters (max(nb0, nb1) / nbpc of
// op.sap_cls CTAs) can be resident at once on this device.
size_t coarse_sap_persist_smem(const CoarseOp<float>& op, int nbpc) {
  if (op.sap_cls <= 0) return 0;
  const int spc = op.g.vB / op.sap_cls;
  return psap_smem_layout(op.g.vB, op.n, spc, op.sap_nsl, nbpc, sizeof(__half2), sizeof(float)).total;
}

namespace {
int persist_threads(const CoarseOp<float>& op, int nbpc) {
  const int spc = op.g.vB / op.sap_cls;
  return ((9 * nbpc * spc * op.n + 31) / 32) * 32;
}
const void* persist_kernel(int nbpc) {
  return nbpc == 2 ? (const void*)k_coarse_sap_persist<float, __half2, 2>
                   : (const void*)k_coarse_sap_persist<float, __half2, 1>;
}
}  // namespace

bool coarse_sap_persist_fits(const CoarseOp<float>& op, int nb0, int nb1, int* max_clusters, int* nbpc_out,
                             int min_nbpc) {
  if (max_clusters) *max_clusters = -1;
  if (nbpc_out) *nbpc_out = 0;
  if (op.sap_cls <= 0 || !op.blkh || nb0 <= 0 || nb1 <= 0) return false;
  const int CLS = op.sap_cls;
  const int nb = nb0 > nb1 ? nb0 : nb1;
  for (int nbpc = min_nbpc < 1 ? 1 : min_nbpc; nbpc <= 2; ++nbpc) {
    const int threads = persist_threads(op, nbpc);
    const size_t sm = coarse_sap_persist_smem(op, nbpc);
    if (threads > 768 || sm > 227 * 1024) continue;
    const void* fn = persist_kernel(nbpc);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             227 * 1024) != cudaSuccess ||   // process-wide limit: the device maximum
        (CLS > 8 && cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)) {
      cudaGetLastError();
      continue;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CLS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(CLS, 1, 1);
    cfg.blockDim = dim3(threads, 1, 1);
    cfg.dynamicSmemBytes = sm;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, fn, &cfg) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (max_clusters) *max_clusters = nclusters;
    if (nclusters >= (nb + nbpc - 1) / nbpc) {
      if (nbpc_out) *nbpc_out = nbpc;
      return true;
    }
  }
  return false;
}

cudaError_t coarse_sap_persist(cplx<float>* z, const cplx<float>* b, const CoarseOp<float>& op, const int* blocks0,
                               int nb0, const int* blocks1, int nb1, int nrhs, size_t rstride, int k_mr, int iters,
                               int nbpc, unsigned* gcnt, cudaStream_t st) {
  if (nrhs <= 0 || iters <= 0) return cudaSuccess;
  if (op.sap_cls <= 0 || !op.blkh || nb0 <= 0 || nb1 <= 0 || nbpc < 1 || nbpc > 2) return cudaErrorInvalidValue;
  const int CLS = op.sap_cls, spc = op.g.vB / CLS;
  const int nb = nb0 > nb1 ? nb0 : nb1;
  cudaError_t e = cudaMemsetAsync(gcnt, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CLS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeCooperative;   // all clusters co-resident (they wait on one another)
  attr[1].val.cooperative = 1;
  cfg.gridDim = dim3(((nb + nbpc - 1) / nbpc) * CLS, 1, 1);
  cfg.blockDim = dim3(persist_threads(op, nbpc), 1, 1);
  cfg.dynamicSmemBytes = coarse_sap_persist_smem(op, nbpc);
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  count_launch();
  if (nbpc == 2)
    return cudaLaunchKernelEx(&cfg, k_coarse_sap_persist<float, __half2, 2>, z, b, op.blkh, op.bscale, op.g, op.n,
                              rstride, nrhs, blocks0, nb0, blocks1, nb1, k_mr, spc, op.sap_nsl, iters, op.err,
                              op.bsite, op.bloc, gcnt);
  return cudaLaunchKernelEx(&cfg, k_coarse_sap_persist<float, __half2, 1>, z, b, op.blkh, op.bscale, op.g, op.n,
                            rstride, nrhs, blocks0, nb0, blocks1, nb1, k_mr, spc, op.sap_nsl, iters, op.err, op.bsite,
                            op.bloc, gcnt);
}

template <typename T>
cudaError_t coarse_sap_sweep(cplx<T>* z, const cplx<T>* b, const CoarseOp<T>& op, const int* blocks, int nblocks,
                             int nrhs, size_t rstride, int k_mr, cudaStream_t st) {
  if (op.sap_cls > 0) {
    const int spc = op.g.vB / op.sap_cls;
    const int threads = ((9 * spc * op.n + 31) / 32) * 32;
    const bool half = sizeof(T) == 4 && op.blkh;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = op.sap_cls;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    // consecutive colour sweeps: the next one stages its blocks while this one finishes
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.gridDim = dim3(nblocks * op.sap_cls, 1, 1);   // one cluster per SAP block loops over the batch
    cfg.blockDim = dim3(threads, 1, 1);
    cfg.dynamicSmemBytes =
        sap_smem_layout(op.g.vB, op.n, spc, op.sap_nsl, half ? sizeof(__half2) : sizeof(cplx<T>), sizeof(T)).total;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    count_launch();
    // with programmatic serialization first, then (if the attribute is refused) without it
    for (int na = 2; na >= 1; --na) {
      cfg.numAttrs = na;
      cudaError_t e;
      if constexpr (sizeof(T) == 4) {
        if (half)
          e = cudaLaunchKernelEx(&cfg, k_coarse_sap_cluster<float, __half2>, z, b, op.blkh, op.bscale, op.g, op.n,
                                 rstride, nrhs, blocks, k_mr, spc, op.sap_nsl, op.err, op.bsite, op.bloc);
        else
          e = cudaLaunchKernelEx(&cfg, k_coarse_sap_cluster<T, cplx<T>>, z, b, (const cplx<T>*)op.blk,
                                 (const float*)nullptr, op.g, op.n, rstride, nrhs, blocks, k_mr, spc, op.sap_nsl,
                                 op.err, op.bsite, op.bloc);
      } else {
        e = cudaLaunchKernelEx(&cfg, k_coarse_sap_cluster<T, cplx<T>>, z, b, (const cplx<T>*)op.blk,
                               (const float*)nullptr, op.g, op.n, rstride, nrhs, blocks, k_mr, spc, op.sap_nsl,
                               op.err, op.bsite, op.bloc);
      }
      if (e == cudaSuccess) return cudaSuccess;
      cudaGetLastError();
    }
    // cluster launch refused: run the one-CTA-per-block kernel instead
  }
  // one CTA per SAP block with rpt rows per thread: the fewest of 1, 4, 8 for which
  // the CTA stays within the threads the kernel's registers allow
  const int rows = op.g.vB * op.n;
  const size_t sm = (size_t)rows * sizeof(cplx<T>) + 32 * 3 * sizeof(T);
  const bool half = sizeof(T) == 4 && op.blkh;
  // threads per CTA the kernel's registers allow, queried once per variant (a property of the
  // compiled kernel, the same on every device of this architecture); the entries are atomics
  // because serving workers launch from several host threads
  static std::atomic<int> maxthr[2][2][3];   // [FP64][FP16 blocks][rpt 1, 4, 8]; 0 = not queried
  std::atomic<int>* mt = maxthr[sizeof(T) == 8][half ? 1 : 0];
  auto query = [&](const void* fn, int q) {
    int v = mt[q].load(std::memory_order_acquire);
    if (v == 0) {
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      cudaFuncAttributes a;
      v = cudaFuncGetAttributes(&a, fn) == cudaSuccess ? a.maxThreadsPerBlock : -1;
      cudaGetLastError();
      mt[q].store(v, std::memory_order_release);
    }
    return v;
  };
  const void* fns[3];
  if constexpr (sizeof(T) == 4) {
    if (half) {
      fns[0] = (const void*)k_coarse_sap<float, __half2, 1>;
      fns[1] = (const void*)k_coarse_sap<float, __half2, 4>;
      fns[2] = (const void*)k_coarse_sap<float, __half2, 8>;
    }
  }
  if (!half) {
    fns[0] = (const void*)k_coarse_sap<T, cplx<T>, 1>;
    fns[1] = (const void*)k_coarse_sap<T, cplx<T>, 4>;
    fns[2] = (const void*)k_coarse_sap<T, cplx<T>, 8>;
  }
  const int rpts[3] = {1, 4, 8};
  int q = 2;
  for (int c = 0; c < 3; ++c)
    if (((div_up(rows, rpts[c]) + 31) / 32) * 32 <= query(fns[c], c)) {
      q = c;
      break;
    }
  const int threads = ((div_up(rows, rpts[q]) + 31) / 32) * 32;
  if (threads > query(fns[q], q)) return cudaErrorInvalidConfiguration;   // block too large even at 8 rows
  count_launch();
  const dim3 grid(nblocks, nrhs);
  if constexpr (sizeof(T) == 4) {
    if (half) {
      if (q == 0)
        k_coarse_sap<float, __half2, 1><<<grid, threads, sm, st>>>(z, b, op.blkh, op.bscale, op.g, op.n, rstride,
                                                                    blocks, k_mr, op.bsite, op.bloc);
      else if (q == 1)
        k_coarse_sap<float, __half2, 4><<<grid, threads, sm, st>>>(z, b, op.blkh, op.bscale, op.g, op.n, rstride,
                                                                    blocks, k_mr, op.bsite, op.bloc);
      else
        k_coarse_sap<float, __half2, 8><<<grid, threads, sm, st>>>(z, b, op.blkh, op.bscale, op.g, op.n, rstride,
                                                                    blocks, k_mr, op.bsite, op.bloc);
      return cudaPeekAtLastError();
    }
  }
  if (q == 0)
    k_coarse_sap<T, cplx<T>, 1><<<grid, threads, sm, st>>>(z, b, op.blk, nullptr, op.g, op.n, rstride, blocks, k_mr,
                                                            op.bsite, op.bloc);
  else if (q == 1)
    k_coarse_sap<T, cplx<T>, 4><<<grid, threads, sm, st>>>(z, b, op.blk, nullptr, op.g, op.n, rstride, blocks, k_mr,
                                                            op.bsite, op.bloc);
  else
    k_coarse_sap<T, cplx<T>, 8><<<grid, threads, sm, st>>>(z, b, op.blk, nullptr, op.g, op.n, rstride, blocks, k_mr,
                                                            op.bsite, op.bloc);
  return cudaPeekAtLastError();
}

template <typename T>
void coarse_schur_odd(cplx<T>* t, const cplx<T>* x, const cplx<T>* b, const CoarseOp<T>& op, double a, double c,
                      int nrhs, size_t rstride, cudaStream_t st) {
  const int threads = ((8 * op.n + 31) / 32) * 32;
  const size_t sm = (size_t)17 * op.n * sizeof(cplx<T>);
  count_launch();
  if constexpr (sizeof(T) == 4) {
    if (op.blkh) {
      k_schur_odd<float, __half2><<<dim3(op.n_odd, nrhs), threads, sm, st>>>(t, x, b, op.blkh, op.bscale, op.selfinv,
                                                                             op.odd_sites, op.g, op.n, rstride, a, c);
      return;
    }
  }
  k_schur_odd<T, cplx<T>><<<dim3(op.n_odd, nrhs), threads, sm, st>>>(t, x, b, op.blk, nullptr, op.selfinv,
                                                                      op.odd_sites, op.g, op.n, rstride, a, c);
}

template <typename T>
void coarse_schur_even(cplx<T>* y, const cplx<T>* x, const cplx<T>* t, const cplx<T>* b, const CoarseOp<T>& op,
                       double a, double s, double c, int nrhs, size_t rstride, cudaStream_t st) {
  const int threads = ((9 * op.n + 31) / 32) * 32;
  const size_t sm = (size_t)18 * op.n * sizeof(cplx<T>);
  count_launch();
  if constexpr (sizeof(T) == 4) {
    if (op.blkh) {
      k_schur_even<float, __half2><<<dim3(op.g.V, nrhs), threads, sm, st>>>(y, x, t, b, op.blkh, op.bscale, op.g, op.n,
                                                                            rstride, a, s, c);
      return;
    }
  }
  k_schur_even<T, cplx<T>><<<dim3(op.g.V, nrhs), threads, sm, st>>>(y, x, t, b, op.blk, nullptr, op.g, op.n, rstride,
                                                                     a, s, c);
}

void coarse_selfinv_build(cplx<double>* inv, const cplx<double>* blk, int V, int n, int* err, cudaStream_t st) {
  const size_t sm = ((size_t)n * 2 * n + n) * sizeof(cplx<double>);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_selfinv_build, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  count_launch();
  k_selfinv_build<<<V, 256, sm, st>>>(inv, blk, n, err);
}

template <typename T>
void coarse_selfinv_apply(cplx<T>* out, const cplx<T>* in, const CoarseOp<T>& op, int parity, int nrhs, size_t rstride,
                          cudaStream_t st) {
  const size_t tot = (size_t)op.g.V * op.n;
  count_launch();
  k_selfinv_apply<T><<<dim3(div_up(tot, 128), nrhs), 128, 0, st>>>(out, in, op.selfinv, op.g, op.n, parity, rstride);
}

template <typename T>
void coarse_sub_parity(cplx<T>* y, const cplx<T>* a, const cplx<T>* b, const Geom& g, int n, int parity, int nrhs,
                       size_t rstride, cudaStream_t st) {
  const size_t tot = (size_t)g.V * n;
  count_launch();
  k_sub_parity<T><<<dim3(div_up(tot, 128), nrhs), 128, 0, st>>>(y, a, b, g, n, parity, rstride);
}

template <typename T>
void coarse_import(cplx<T>* dst, const cplx<double>* src, const Geom& g, int n, int nrhs, size_t rstride,
                   cudaStream_t st) {
  count_launch();
  k_coarse_import<T><<<dim3(div_up((size_t)g.V * n, 128), nrhs), 128, 0, st>>>(dst, src, g, n, rstride);
}

template <typename T>
void coarse_export(cplx<double>* dst, const cplx<T>* src, const Geom& g, int n, int nrhs, size_t rstride,
                   cudaStream_t st) {
  count_launch();
  k_coarse_export<T><<<dim3(div_up((size_t)g.V * n, 128), nrhs), 128, 0, st>>>(dst, src, g, n, rstride);
}

void coarse_blocks_export(cplx<double>* dst, const cplx<double>* blk, const Geom& g, int n, cudaStream_t st) {
  count_launch();
  k_blocks_export<<<div_up((size_t)g.V * 9 * n * n, 128), 128, 0, st>>>(dst, blk, g, n);
}

#define INST(T)                                                                                                   \
  template void coarse_apply<T>(cplx<T>*, const cplx<T>*, const cplx<T>*, const CoarseOp<T>&, int, size_t, int,     \
                                int, int, cudaStream_t);                                                          \
  template void coarse_schur_odd<T>(cplx<T>*, const cplx<T>*, const cplx<T>*, const CoarseOp<T>&, double, double, \
                                    int, size_t, cudaStream_t);                                                   \
  template void coarse_schur_even<T>(cplx<T>*, const cplx<T>*, const cplx<T>*, const cplx<T>*, const CoarseOp<T>&, \
                                     double, double, double, int, size_t, cudaStream_t);                          \
  template int coarse_sap_cluster_plan<T>(const Geom&, int, int*, int*, int*, int);                                \
  template cudaError_t coarse_sap_sweep<T>(cplx<T>*, const cplx<T>*, const CoarseOp<T>&, const int*, int, int, size_t,   \
                                    int, cudaStream_t);                                                           \
  template void coarse_selfinv_apply<T>(cplx<T>*, const cplx<T>*, const CoarseOp<T>&, int, int, size_t,           \
                                        cudaStream_t);                                                            \
  template void coarse_sub_parity<T>(cplx<T>*, const cplx<T>*, const cplx<T>*, const Geom&, int, int, int, size_t, \
                                     cudaStream_t);                                                               \
  template void coarse_import<T>(cplx<T>*, const cplx<double>*, const Geom&, int, int, size_t, cudaStream_t);      \
  template void coarse_export<T>(cplx<double>*, const cplx<T>*, const Geom&, int, int, size_t, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace dd
