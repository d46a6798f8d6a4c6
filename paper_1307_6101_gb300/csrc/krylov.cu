// Device-driven (F)GMRES for the inner solves of the K-cycle (Alg. 2) and the
// coarsest odd-even GMRES, so that one whole preconditioner application can be
// captured into a CUDA graph whose Krylov loops are conditional WHILE nodes.
//
// Arithmetic is the same as the host-driven solver: Arnoldi with classical
// Gram-Schmidt applied twice, Givens rotations, per-right-hand-side stopping
// (|g_{j+1}| <= tol ||b|| inside a cycle, true residual between cycles).  Each
// right-hand side is handled by its own CTA (or its own cluster, for long
// vectors) in the fused Arnoldi step, so the reduction order of a right-hand
// side does not depend on the batch.  Loop
// conditions are set by the last CTA to finish (atomic arrival counter, no
// waiting); every loop is bounded by its maximal iteration count.
#include "common.cuh"
#include "kernels.h"

#include <cooperative_groups.h>

namespace cg = cooperative_groups;

namespace {

constexpr int AT = 512;   // threads of the fused Arnoldi CTA

template <typename A>
__device__ A block_sum_d(A v, A* sh) {
  for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  A s = A(0);
  for (int w = 0; w < nw; ++w) s += sh[w];
  return s;
}

// sum 16 values per thread over the CTA; results in sh_out[0..15] (valid after return)
template <typename A>
__device__ void block_sum16(A* v, A* sh, A* sh_out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int k = 0; k < 16; ++k)
    for (int off = 16; off >= 1; off >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], off);
  __syncthreads();
  if (lane == 0)
    for (int k = 0; k < 16; ++k) sh[warp * 16 + k] = v[k];
  __syncthreads();
  if (threadIdx.x < 16) {
    A s = A(0);
    for (int w = 0; w < nw; ++w) s += sh[w * 16 + threadIdx.x];
    sh_out[threadIdx.x] = s;
  }
  __syncthreads();
}

// last CTA to arrive returns true (arrival counter reset for the next launch)
__device__ bool last_block(int* counter, int nblocks) {
  __shared__ int is_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const int t = atomicAdd(counter, 1);
    is_last = (t == nblocks - 1);
    if (is_last) *counter = 0;
  }
  __syncthreads();
  if (is_last) __threadfence();
  return is_last != 0;
}

__global__ void k_kry_start(dd::GmresState s, int nrhs, double tol, cudaGraphConditionalHandle hcycle) {
  if (threadIdx.x == 0) {
    s.ctl[0] = 0;   // j
    s.ctl[1] = 0;   // cycle
    s.ctl[2] = 0;   // arrival counter
  }
  for (int r = threadIdx.x; r < nrhs; r += blockDim.x) {
    const double b = s.beta[r];
    s.bnorm[r] = b;
    s.target[r] = tol * b;
    s.conv[r] = (b <= tol * b) ? 1 : 0;
    s.iters[r] = 0;
  }
  if (threadIdx.x == 0) cudaGraphSetConditional(hcycle, 1u);
}

// begin a restart cycle: g = beta e1, V_0 = r / beta, cur = V_0.  gridDim.x
// CTAs per rhs share the scaling; CTA 0 of a rhs writes its state.
template <typename T>
__global__ void k_cycle_begin(dd::GmresState s, cplx<T>* __restrict__ V0, cplx<T>* __restrict__ cur,
                              const cplx<T>* __restrict__ r, size_t vlen, size_t rstride, int nrhs,
                              cudaGraphConditionalHandle hinner) {
  const int rh = blockIdx.y;
  const int m = s.m;
  const double b = s.beta[rh];
  const int dn = (s.conv[rh] || b <= s.target[rh]) ? 1 : 0;
  const double inv = (dn || b == 0.0) ? 0.0 : 1.0 / b;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    s.done[rh] = dn;
    s.inv[rh] = inv;
    s.kr[rh] = 0;
    s.est[rh] = b;
    for (int k = 0; k <= m; ++k) s.g[(size_t)rh * (m + 1) + k] = czero<double>();
    s.g[(size_t)rh * (m + 1)] = cmk(b, 0.0);
    for (int k = 0; k < m; ++k) s.y[(size_t)rh * m + k] = czero<double>();
  }
  const T iv = (T)inv;
  const size_t o = (size_t)rh * rstride;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < vlen; e += (size_t)gridDim.x * blockDim.x) {
    const cplx<T> v = iv * r[o + e];
    V0[o + e] = v;
    cur[o + e] = v;
  }
  if (last_block(s.ctl + 2, nrhs * gridDim.x) && threadIdx.x == 0) {
    s.ctl[0] = 0;
    int any = 0;
    for (int q = 0; q < nrhs; ++q) any |= !((volatile int*)s.done)[q];
    cudaGraphSetConditional(hinner, any ? 1u : 0u);
  }
}

// column j of the Hessenberg matrix of rhs rh from h_0..h_j (htot) and ||w||^2 = nn:
// previous rotations, the new rotation, residual estimate and stopping flag;
// returns 1/||w|| (0 when the rhs stops)
__device__ double givens_column(dd::GmresState& s, int rh, int j, const cplx<double>* htot, double nn) {
  const int m = s.m;
  cplx<double>* H = s.H + (size_t)rh * (m + 1) * m;
  cplx<double>* g = s.g + (size_t)rh * (m + 1);
  double* cs = s.cs + (size_t)rh * m;
  cplx<double>* sn = s.sn + (size_t)rh * m;
  const double hn = sqrt(nn);
  cplx<double> h[65];
  for (int i = 0; i <= j; ++i) h[i] = htot[i];
  h[j + 1] = cmk(hn, 0.0);
  for (int i = 0; i < j; ++i) {
    const cplx<double> t = cs[i] * h[i] + sn[i] * h[i + 1];
    h[i + 1] = cs[i] * h[i + 1] - cconj(sn[i]) * h[i];
    h[i] = t;
  }
  // rotation zeroing h[j+1]
  const double aa = sqrt(cnorm2(h[j])), bb = sqrt(cnorm2(h[j + 1]));
  const double rr = hypot(aa, bb);
  double c;
  cplx<double> sg;
  if (rr == 0.0) { c = 1.0; sg = czero<double>(); }
  else if (aa == 0.0) { c = 0.0; sg = bb == 0.0 ? cmk(1.0, 0.0) : cmk(h[j + 1].re / bb, -h[j + 1].im / bb); }
  else {
    c = aa / rr;
    const cplx<double> ph = cmk(h[j].re / aa, h[j].im / aa);
    sg = (1.0 / rr) * (ph * cconj(h[j + 1]));
  }
  cs[j] = c;
  sn[j] = sg;
  h[j] = c * h[j] + sg * h[j + 1];
  h[j + 1] = czero<double>();
  g[j + 1] = -1.0 * (cconj(sg) * g[j]);
  g[j] = c * g[j];
  for (int i = 0; i <= j + 1; ++i) H[(size_t)i * m + j] = h[i];
  s.kr[rh] = j + 1;
  const double est = sqrt(cnorm2(g[j + 1]));
  s.est[rh] = est;
  double inv = hn > 0.0 ? 1.0 / hn : 0.0;
  if (est <= s.target[rh] || hn == 0.0 || j + 1 == m) {
    s.done[rh] = 1;
    inv = 0.0;
  }
  s.inv[rh] = inv;
  return inv;
}

// the last of nblocks CTAs advances j and sets the Arnoldi loop condition
__device__ void arnoldi_advance(dd::GmresState& s, int nrhs, int nblocks, int j, int m,
                                cudaGraphConditionalHandle hinner) {
  if (last_block(s.ctl + 2, nblocks) && threadIdx.x == 0) {
    const int jn = j + 1;
    s.ctl[0] = jn;
    s.ctl[3] += 1;   // Arnoldi steps of this solver since setup (diagnostics)
    int any = 0;
    for (int q = 0; q < nrhs; ++q) any |= !((volatile int*)s.done)[q];
    cudaGraphSetConditional(hinner, (any && jn < m) ? 1u : 0u);
  }
}

// One Arnoldi step for every rhs (one CTA each; long vectors use the cluster
// variant k_arnoldi_cl below): CGS2 of w against V_0..V_j,
// ||w||, Givens update of column j, V_{j+1} = w / ||w||, cur = V_{j+1},
// Z_j = zcur (flexible).  The last CTA advances j and sets the loop condition.
template <typename T>
__global__ void __launch_bounds__(AT) k_arnoldi(dd::GmresState s, cplx<T>* __restrict__ V, size_t vstride,
                                                cplx<T>* __restrict__ Z, const cplx<T>* __restrict__ zcur,
                                                cplx<T>* __restrict__ w, cplx<T>* __restrict__ cur, size_t vlen,
                                                size_t rstride, int nrhs, cudaGraphConditionalHandle hinner) {
  // reductions run in the precision of the vectors: FP32 data is summed in FP32
  // (tree order), FP64 data in FP64; the Hessenberg/Givens updates are FP64
  __shared__ T sh[32 * 16];
  __shared__ T red[16];
  __shared__ cplx<double> hs[64];
  __shared__ cplx<double> htot[64];
  __shared__ double inv_s;
  const int rh = blockIdx.x;
  const int m = s.m;
  const int j = ((volatile int*)s.ctl)[0];
  const size_t o = (size_t)rh * rstride;
  cplx<T>* pw = w + o;
  const bool dn = s.done[rh] != 0;
  if (!dn) {
    for (int i = threadIdx.x; i <= j; i += blockDim.x) htot[i] = czero<double>();
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
      for (int i0 = 0; i0 <= j; i0 += 8) {
        T acc[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) acc[k] = T(0);
        for (size_t e = threadIdx.x; e < vlen; e += blockDim.x) {
          const cplx<T> we = pw[e];
#pragma unroll
          for (int ii = 0; ii < 8; ++ii) {
            if (i0 + ii <= j) {
              const cplx<T> v = V[(size_t)(i0 + ii) * vstride + o + e];
              acc[2 * ii] += v.re * we.re + v.im * we.im;
              acc[2 * ii + 1] += v.re * we.im - v.im * we.re;
            }
          }
        }
        block_sum16<T>(acc, sh, red);
        if (threadIdx.x < 8 && i0 + threadIdx.x <= j) {
          const cplx<double> hv = cmk((double)red[2 * threadIdx.x], (double)red[2 * threadIdx.x + 1]);
          hs[i0 + threadIdx.x] = hv;
          htot[i0 + threadIdx.x] = htot[i0 + threadIdx.x] + hv;
        }
        __syncthreads();
      }
      for (size_t e = threadIdx.x; e < vlen; e += blockDim.x) {
        cplx<T> we = pw[e];
        for (int i = 0; i <= j; ++i) {
          const cplx<T> c = cmk<T>((T)hs[i].re, (T)hs[i].im);
          we = we - c * V[(size_t)i * vstride + o + e];
        }
        pw[e] = we;
      }
      __syncthreads();
    }
    T nnt = T(0);
    for (size_t e = threadIdx.x; e < vlen; e += blockDim.x) nnt += cnorm2(pw[e]);
    const double nn = (double)block_sum_d<T>(nnt, sh);
    if (threadIdx.x == 0) inv_s = givens_column(s, rh, j, htot, nn);
  } else if (threadIdx.x == 0) {
    s.inv[rh] = 0.0;
    inv_s = 0.0;
  }
  __syncthreads();
  const T iv = (T)inv_s;
  cplx<T>* vn = V + (size_t)(j + 1) * vstride + o;
  for (size_t e = threadIdx.x; e < vlen; e += blockDim.x) {
    const cplx<T> v = iv * pw[e];
    vn[e] = v;
    cur[o + e] = v;
    if (Z) Z[(size_t)j * vstride + o + e] = zcur[o + e];
  }
  arnoldi_advance(s, nrhs, nrhs, j, m, hinner);
}

// The same Arnoldi step for long vectors: a cluster of gridDim.x CTAs per rhs
// (blockIdx.y), CTA q owning the contiguous slice q of the vector.  The partial
// sums of each batch of eight dots (and of ||w||^2) go to the CTA's shared
// memory; after a cluster barrier every CTA adds the partials of all ranks in
// rank order, so all CTAs hold the same h and the result does not depend on the
// batch.  The partial buffers alternate between batches, so one barrier per
// batch suffices.  Rank 0 updates the Givens rotations and broadcasts 1/||w||.
template <typename T>
__global__ void __launch_bounds__(AT) k_arnoldi_cl(dd::GmresState s, cplx<T>* __restrict__ V, size_t vstride,
                                                   cplx<T>* __restrict__ Z, const cplx<T>* __restrict__ zcur,
                                                   cplx<T>* __restrict__ w, cplx<T>* __restrict__ cur, size_t vlen,
                                                   size_t rstride, int nrhs, cudaGraphConditionalHandle hinner) {
  cg::cluster_group cl = cg::this_cluster();
  __shared__ T sh[32 * 16];
  __shared__ T red[16];
  __shared__ T part[2][16];
  __shared__ cplx<double> hs[64];
  __shared__ cplx<double> htot[64];
  __shared__ double inv_s;
  const int CL = (int)cl.num_blocks();
  const int q = (int)cl.block_rank();
  const int rh = blockIdx.y;
  const int m = s.m;
  const int j = ((volatile int*)s.ctl)[0];
  const size_t o = (size_t)rh * rstride;
  const size_t per = (vlen + CL - 1) / CL;
  const size_t lo = (size_t)q * per < vlen ? (size_t)q * per : vlen;
  const size_t hi = lo + per < vlen ? lo + per : vlen;
  cplx<T>* pw = w + o;
  const bool dn = s.done[rh] != 0;   // the same for every CTA of the cluster
  if (!dn) {
    int batch = 0;
    for (int i = threadIdx.x; i <= j; i += blockDim.x) htot[i] = czero<double>();
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
      for (int i0 = 0; i0 <= j; i0 += 8, ++batch) {
        T acc[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) acc[k] = T(0);
        for (size_t e = lo + threadIdx.x; e < hi; e += blockDim.x) {
          const cplx<T> we = pw[e];
#pragma unroll
          for (int ii = 0; ii < 8; ++ii) {
            if (i0 + ii <= j) {
              const cplx<T> v = V[(size_t)(i0 + ii) * vstride + o + e];
              acc[2 * ii] += v.re * we.re + v.im * we.im;
              acc[2 * ii + 1] += v.re * we.im - v.im * we.re;
            }
          }
        }
        block_sum16<T>(acc, sh, red);
        if (threadIdx.x < 16) part[batch & 1][threadIdx.x] = red[threadIdx.x];
        cl.sync();
        if (threadIdx.x < 8 && i0 + threadIdx.x <= j) {
          T re = T(0), im = T(0);
          for (int r = 0; r < CL; ++r) {
            const T* pr = cl.map_shared_rank(&part[batch & 1][0], r);
            re += pr[2 * threadIdx.x];
            im += pr[2 * threadIdx.x + 1];
          }
          const cplx<double> hv = cmk((double)re, (double)im);
          hs[i0 + threadIdx.x] = hv;
          htot[i0 + threadIdx.x] = htot[i0 + threadIdx.x] + hv;
        }
        __syncthreads();
      }
      for (size_t e = lo + threadIdx.x; e < hi; e += blockDim.x) {
        cplx<T> we = pw[e];
        for (int i = 0; i <= j; ++i) {
          const cplx<T> c = cmk<T>((T)hs[i].re, (T)hs[i].im);
          we = we - c * V[(size_t)i * vstride + o + e];
        }
        pw[e] = we;
      }
      __syncthreads();
    }
    T nnt = T(0);
    for (size_t e = lo + threadIdx.x; e < hi; e += blockDim.x) nnt += cnorm2(pw[e]);
    const T nnq = block_sum_d<T>(nnt, sh);
    if (threadIdx.x == 0) part[batch & 1][0] = nnq;
    cl.sync();
    if (q == 0 && threadIdx.x == 0) {
      T nn = T(0);
      for (int r = 0; r < CL; ++r) nn += *cl.map_shared_rank(&part[batch & 1][0], r);
      inv_s = givens_column(s, rh, j, htot, (double)nn);
    }
    cl.sync();
    if (threadIdx.x == 0) inv_s = *cl.map_shared_rank(&inv_s, 0);
    cl.sync();   // rank 0's shared memory is read before any CTA leaves
  } else if (threadIdx.x == 0) {
    if (q == 0) s.inv[rh] = 0.0;
    inv_s = 0.0;
  }
  __syncthreads();
  const T iv = (T)inv_s;
  cplx<T>* vn = V + (size_t)(j + 1) * vstride + o;
  for (size_t e = lo + threadIdx.x; e < hi; e += blockDim.x) {
    const cplx<T> v = iv * pw[e];
    vn[e] = v;
    cur[o + e] = v;
    if (Z) Z[(size_t)j * vstride + o + e] = zcur[o + e];
  }
  arnoldi_advance(s, nrhs, nrhs * CL, j, m, hinner);
}

__global__ void k_cycle_end(dd::GmresState s, int nrhs, int max_cycles, cudaGraphConditionalHandle hcycle) {
  if (threadIdx.x != 0) return;
  const int cycle = ++s.ctl[1];
  int any = 0;
  for (int r = 0; r < nrhs; ++r) {
    if (!s.conv[r]) {
      s.iters[r] += s.kr[r];
      if (s.beta[r] <= s.target[r]) s.conv[r] = 1;
    }
    any |= !s.conv[r];
  }
  cudaGraphSetConditional(hcycle, (any && cycle < max_cycles) ? 1u : 0u);
}

}  // namespace

namespace dd {

void kry_start(const GmresState& s, int nrhs, double tol, cudaGraphConditionalHandle hcycle, cudaStream_t st) {
  count_launch();
  k_kry_start<<<1, 128, 0, st>>>(s, nrhs, tol, hcycle);
}

template <typename T>
void kry_cycle_begin(const GmresState& s, cplx<T>* V0, cplx<T>* cur, const cplx<T>* r, size_t vlen, int nrhs,
                     cudaGraphConditionalHandle hinner, cudaStream_t st) {
  size_t nb = (vlen + 8191) / 8192;   // CTAs per rhs
  if (nb > 16) nb = 16;
  count_launch();
  k_cycle_begin<T><<<dim3((unsigned)nb, nrhs), 256, 0, st>>>(s, V0, cur, r, vlen, vlen, nrhs, hinner);
}

// cluster size of the split Arnoldi step for vectors of length vlen: about 1024
// elements per CTA, at most 16 (8 if the device cannot co-schedule 16); 1 = one CTA
template <typename T>
int arnoldi_cluster(size_t vlen) {
  static int cmax = -1;
  if (cmax < 0) {
    cmax = 1;
    for (int c : {16, 8}) {
      if (c > 8 && cudaFuncSetAttribute(k_arnoldi_cl<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                       cudaSuccess) {
        cudaGetLastError();
        continue;
      }
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = c;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3(c, 1, 1);
      cfg.blockDim = dim3(AT, 1, 1);
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      int n = 0;
      if (cudaOccupancyMaxActiveClusters(&n, k_arnoldi_cl<T>, &cfg) == cudaSuccess && n >= 1) {
        cmax = c;
        break;
      }
      cudaGetLastError();
    }
  }
  int c = 1;
  while (c < cmax && vlen >= (size_t)2048 * c) c <<= 1;
  return c;
}

template <typename T>
cudaError_t kry_arnoldi(const GmresState& s, cplx<T>* V, size_t vstride, cplx<T>* Z, const cplx<T>* zcur, cplx<T>* w,
                        cplx<T>* cur, size_t vlen, int nrhs, cudaGraphConditionalHandle hinner, cudaStream_t st) {
  const int c = arnoldi_cluster<T>(vlen);
  count_launch();
  if (c == 1) {
    k_arnoldi<T><<<nrhs, AT, 0, st>>>(s, V, vstride, Z, zcur, w, cur, vlen, vlen, nrhs, hinner);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = c;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(c, nrhs, 1);
  cfg.blockDim = dim3(AT, 1, 1);
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_arnoldi_cl<T>, s, V, vstride, Z, zcur, w, cur, vlen, (size_t)vlen, nrhs, hinner);
}

void kry_prepare() {
  arnoldi_cluster<float>(0);
  arnoldi_cluster<double>(0);
}

void kry_cycle_end(const GmresState& s, int nrhs, int max_cycles, cudaGraphConditionalHandle hcycle, cudaStream_t st) {
  count_launch();
  k_cycle_end<<<1, 32, 0, st>>>(s, nrhs, max_cycles, hcycle);
}

#define INST(T)                                                                                                  \
  template void kry_cycle_begin<T>(const GmresState&, cplx<T>*, cplx<T>*, const cplx<T>*, size_t, int,           \
                                   cudaGraphConditionalHandle, cudaStream_t);                                    \
  template cudaError_t kry_arnoldi<T>(const GmresState&, cplx<T>*, size_t, cplx<T>*, const cplx<T>*, cplx<T>*,    \
                                      cplx<T>*, size_t, int, cudaGraphConditionalHandle, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace dd
