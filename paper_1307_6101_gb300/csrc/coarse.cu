// Coarse-level kernels: the Galerkin operators D_{l+1} = P_l^+ D_l P_l are
// nearest-neighbour stencils of dense n x n complex blocks (Sec. 1, Sec. 2):
//   (D phi)(A) = S(A) phi(A) + sum_mu [ F_mu(A) phi(A + mu) + B_mu(A) phi(A - mu) ].
// Blocks are stored column-major per (site, k) with k = 0 self, 1..4 forward,
// 5..8 backward, so that the threads computing consecutive rows of one site
// read consecutive words.
#include "common.cuh"
#include "kernels.h"

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

template <typename T, bool RESID>
__global__ void k_coarse_apply(cplx<T>* __restrict__ out, const cplx<T>* __restrict__ in,
                               const cplx<T>* __restrict__ bsrc, const cplx<T>* __restrict__ blk, Geom g, int n,
                               size_t rstride, int sel, int sel_mu, int in_chir) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)g.V * n) return;
  const int site = (int)(t / n), i = (int)(t % n);
  const size_t ro = (size_t)blockIdx.y * rstride;
  const cplx<T>* pin = in + ro;
  int c[4];
  geom_coords(g, site, c);
  const int h = n / 2;
  const int j0 = in_chir == 1 ? h : 0;
  const int j1 = in_chir == 0 ? h : n;
  cplx<T> acc = czero<T>();
  if (sel == SEL_FULL || sel == SEL_AGG_SELF) {
    const cplx<T>* v = pin + (size_t)site * n;
    for (int j = j0; j < j1; ++j) cfma(acc, blk[bidx(site, 0, n, i, j)], v[j]);
  }
  for (int mu = 0; mu < 4; ++mu) {
    const bool inf = hop_internal(g, c, mu, +1, g.A);
    const bool inb = hop_internal(g, c, mu, -1, g.A);
    bool tf = true, tb = true;
    if (sel == SEL_AGG_SELF) { tf = inf; tb = inb; }
    else if (sel == SEL_AGG_FWD) { tf = (mu == sel_mu) && !inf; tb = false; }
    else if (sel == SEL_AGG_BWD) { tf = false; tb = (mu == sel_mu) && !inb; }
    if (tf) {
      const cplx<T>* v = pin + (size_t)geom_neighbor(g, c, mu, +1) * n;
      for (int j = j0; j < j1; ++j) cfma(acc, blk[bidx(site, 1 + mu, n, i, j)], v[j]);
    }
    if (tb) {
      const cplx<T>* v = pin + (size_t)geom_neighbor(g, c, mu, -1) * n;
      for (int j = j0; j < j1; ++j) cfma(acc, blk[bidx(site, 5 + mu, n, i, j)], v[j]);
    }
  }
  if (RESID) out[ro + t] = bsrc[ro + t] - acc;
  else out[ro + t] = acc;
}

// One colour sweep of SAP on a coarse level: one CTA per SAP block, one thread
// per (site, row) of the block.  rho = (b - D z)_B, k MR steps on D_B, z_B += e_B.
template <typename T>
__global__ void k_coarse_sap(cplx<T>* __restrict__ z, const cplx<T>* __restrict__ bsrc,
                             const cplx<T>* __restrict__ blk, Geom g, int n, size_t rstride,
                             const int* __restrict__ blocks, int k_mr) {
  extern __shared__ unsigned char smem_raw[];
  cplx<T>* rs = reinterpret_cast<cplx<T>*>(smem_raw);        // [vB * n]
  T* sh = reinterpret_cast<T*>(rs + (size_t)g.vB * n);          // [warps][3]
  const int b = blocks[blockIdx.x];
  const int loc = threadIdx.x / n, i = threadIdx.x % n;
  const bool active = loc < g.vB;
  const int site = b * g.vB + (active ? loc : 0);
  const size_t ro = (size_t)blockIdx.y * rstride;
  cplx<T>* pz = z + ro;
  int c[4];
  geom_coords(g, site, c);
  cplx<T> r = czero<T>(), xs = czero<T>();
  if (active) {
    cplx<T> acc = czero<T>();
    const cplx<T>* v = pz + (size_t)site * n;
    for (int j = 0; j < n; ++j) cfma(acc, blk[bidx(site, 0, n, i, j)], v[j]);
    for (int mu = 0; mu < 4; ++mu) {
      v = pz + (size_t)geom_neighbor(g, c, mu, +1) * n;
      for (int j = 0; j < n; ++j) cfma(acc, blk[bidx(site, 1 + mu, n, i, j)], v[j]);
      v = pz + (size_t)geom_neighbor(g, c, mu, -1) * n;
      for (int j = 0; j < n; ++j) cfma(acc, blk[bidx(site, 5 + mu, n, i, j)], v[j]);
    }
    r = bsrc[ro + (size_t)site * n + i] - acc;
  }
  for (int it = 0; it < k_mr; ++it) {
    if (active) rs[threadIdx.x] = r;
    __syncthreads();
    T nre = T(0), nim = T(0), den = T(0);
    cplx<T> p = czero<T>();
    if (active) {
      const cplx<T>* v = rs + (size_t)loc * n;
      for (int j = 0; j < n; ++j) cfma(p, blk[bidx(site, 0, n, i, j)], v[j]);
      for (int mu = 0; mu < 4; ++mu) {
        if (hop_internal(g, c, mu, +1, g.B)) {
          const int nl = geom_neighbor(g, c, mu, +1) - b * g.vB;
          v = rs + (size_t)nl * n;
          for (int j = 0; j < n; ++j) cfma(p, blk[bidx(site, 1 + mu, n, i, j)], v[j]);
        }
        if (hop_internal(g, c, mu, -1, g.B)) {
          const int nl = geom_neighbor(g, c, mu, -1) - b * g.vB;
          v = rs + (size_t)nl * n;
          for (int j = 0; j < n; ++j) cfma(p, blk[bidx(site, 5 + mu, n, i, j)], v[j]);
        }
      }
      const cplx<T> tt = cdotc(p, r);
      nre = tt.re;
      nim = tt.im;
      den = cnorm2(p);
    }
    cta_sum3(nre, nim, den, sh);
    const cplx<T> alpha = den > T(0) ? cmk<T>(nre / den, nim / den) : czero<T>();
    cfma(xs, alpha, r);
    r = r - alpha * p;
  }
  if (active) {
    const size_t a = ro + (size_t)site * n + i;
    z[a] = z[a] + xs;
  }
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

}  // namespace

namespace dd {

template <typename T>
void coarse_apply(cplx<T>* out, const cplx<T>* in, const cplx<T>* b, const CoarseOp<T>& op, int nrhs, size_t rstride,
                  int sel, int sel_mu, int in_chir, cudaStream_t st) {
  const size_t tot = (size_t)op.g.V * op.n;
  dim3 grid(div_up(tot, 128), nrhs);
  if (b)
    k_coarse_apply<T, true><<<grid, 128, 0, st>>>(out, in, b, op.blk, op.g, op.n, rstride, sel, sel_mu, in_chir);
  else
    k_coarse_apply<T, false><<<grid, 128, 0, st>>>(out, in, b, op.blk, op.g, op.n, rstride, sel, sel_mu, in_chir);
}

template <typename T>
void coarse_sap_sweep(cplx<T>* z, const cplx<T>* b, const CoarseOp<T>& op, const int* blocks, int nblocks, int nrhs,
                      size_t rstride, int k_mr, cudaStream_t st) {
  const int threads = ((op.g.vB * op.n + 31) / 32) * 32;
  const size_t sm = (size_t)op.g.vB * op.n * sizeof(cplx<T>) + 32 * 3 * sizeof(T);
  static bool attr_set[2] = {false, false};
  bool& done = attr_set[sizeof(T) == 8];
  if (!done) {
    cudaFuncSetAttribute(k_coarse_sap<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    done = true;
  }
  k_coarse_sap<T><<<dim3(nblocks, nrhs), threads, sm, st>>>(z, b, op.blk, op.g, op.n, rstride, blocks, k_mr);
}

void coarse_selfinv_build(cplx<double>* inv, const cplx<double>* blk, int V, int n, int* err, cudaStream_t st) {
  const size_t sm = ((size_t)n * 2 * n + n) * sizeof(cplx<double>);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_selfinv_build, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  k_selfinv_build<<<V, 256, sm, st>>>(inv, blk, n, err);
}

template <typename T>
void coarse_selfinv_apply(cplx<T>* out, const cplx<T>* in, const CoarseOp<T>& op, int parity, int nrhs, size_t rstride,
                          cudaStream_t st) {
  const size_t tot = (size_t)op.g.V * op.n;
  k_selfinv_apply<T><<<dim3(div_up(tot, 128), nrhs), 128, 0, st>>>(out, in, op.selfinv, op.g, op.n, parity, rstride);
}

template <typename T>
void coarse_sub_parity(cplx<T>* y, const cplx<T>* a, const cplx<T>* b, const Geom& g, int n, int parity, int nrhs,
                       size_t rstride, cudaStream_t st) {
  const size_t tot = (size_t)g.V * n;
  k_sub_parity<T><<<dim3(div_up(tot, 128), nrhs), 128, 0, st>>>(y, a, b, g, n, parity, rstride);
}

template <typename T>
void coarse_import(cplx<T>* dst, const cplx<double>* src, const Geom& g, int n, int nrhs, size_t rstride,
                   cudaStream_t st) {
  k_coarse_import<T><<<dim3(div_up((size_t)g.V * n, 128), nrhs), 128, 0, st>>>(dst, src, g, n, rstride);
}

template <typename T>
void coarse_export(cplx<double>* dst, const cplx<T>* src, const Geom& g, int n, int nrhs, size_t rstride,
                   cudaStream_t st) {
  k_coarse_export<T><<<dim3(div_up((size_t)g.V * n, 128), nrhs), 128, 0, st>>>(dst, src, g, n, rstride);
}

void coarse_blocks_export(cplx<double>* dst, const cplx<double>* blk, const Geom& g, int n, cudaStream_t st) {
  k_blocks_export<<<div_up((size_t)g.V * 9 * n * n, 128), 128, 0, st>>>(dst, blk, g, n);
}

#define INST(T)                                                                                                   \
  template void coarse_apply<T>(cplx<T>*, const cplx<T>*, const cplx<T>*, const CoarseOp<T>&, int, size_t, int,     \
                                int, int, cudaStream_t);                                                          \
  template void coarse_sap_sweep<T>(cplx<T>*, const cplx<T>*, const CoarseOp<T>&, const int*, int, int, size_t,   \
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
