// Internal launch API of the DD-alpha-AMG CUDA library (not part of the C ABI).
#pragma once

#include "common.cuh"
#include "dfloat.cuh"

namespace dd {

// number of kernels this library has launched (all streams, all handles)
void count_launch(int k = 1);
long long launch_count();

template <typename T>
struct FineOp {
  Geom g;
  int bc_t;
  cplx<T>* U;    // [4][9][V]
  T* clov;       // [2][36][V]  (m0 + 4) + clover, packed Hermitian
  int* err;      // device error flag (bounded waits), may be null
  // FP16 storage (FP32 compute only): when Uh is set the kernels read these instead
  const __half2* Uh = nullptr;   // [4][9][V] links
  const __half2* clovh = nullptr; // [2][18][V] clover term without the (m0 + 4) shift, pairs of packed reals
  float shift = 0.f;             // m0 + 4, added to the diagonal in FP32
  // SAP block solves on the even-odd Schur complement (FP32 compute, 4^4 blocks): per-site tables
  // with the clover term on even sites and the inverse of (m0 + 4) + clover on odd sites
  bool schur = false;
  const float* mix32 = nullptr;    // [2][36][V] (even sites with the shift)
  const __half2* mixh = nullptr;   // [2][18][V] (even sites without the shift)
};

template <typename T>
struct CoarseOp {
  Geom g;
  int n;                // dof per site
  cplx<T>* blk;         // [V][9][n][n] column-major blocks
  cplx<T>* selfinv;     // [V][n][n] inverse of the self block (coarsest level), or null
  const int* odd_sites; // indices of the odd sites (coarsest level), or null
  int n_odd;
  int sap_cls;          // cluster size of the cluster SAP kernel (0: one CTA per SAP block)
  int sap_nsl = 0;      // blocks per site staged in shared memory by the cluster SAP kernel
  const int* bsite = nullptr;   // [nBlk][vB] sites of each SAP block (block-local order)
  const int* bloc = nullptr;    // [V] position of each site inside its SAP block
  int* err = nullptr;   // device error flag (bounded waits)
  // FP16 storage (FP32 compute only): blocks and one scale per site
  const __half2* blkh = nullptr;
  const float* bscale = nullptr;
  // full applications on FP16 storage: 0 = CUDA-core kernel, k >= 1 = tensor-core kernel with the
  // k-dimension split over k warp groups (chosen per level by the autotuner)
  int tc_ks = 0;
};

// ---- fine level -----------------------------------------------------------
void set_gamma_products(const double* gg);
template <typename T>
void fine_dslash(cplx<T>* out, const cplx<T>* in, const cplx<T>* b, const FineOp<T>& op, int nrhs, size_t rstride,
                 int sel, int sel_mu, int in_chir, cudaStream_t st);
template <typename T>
void fine_sap_sweep(cplx<T>* z, const cplx<T>* b, const FineOp<T>& op, const int* blocks, int nblocks, int nrhs,
                    size_t rstride, int k_mr, cudaStream_t st);
// ||b_i - D x_i|| / ||b_i|| with FP64 b, x in the ABI layout (device memory), no
// allocation (static scratch); returns 0 or a negative code with *msg set
int fine_residual_norm_noalloc(double* out, bool out_on_device, const cplx<double>* b, const cplx<double>* x,
                               const FineOp<double>& op, int device, int nrhs, cudaStream_t st, const char** msg);
void clover_build(double* clov, const cplx<double>* gauge_lex, const Geom& g, double m0, double csw,
                  cudaStream_t st);
// out = Gamma_5 in on nrhs fine FP64 fields (may be in place)
void fine_gamma5(cplx<double>* out, const cplx<double>* in, int V, int nrhs, size_t rstride, cudaStream_t st);
// double-FP32 operator data (pairs rounded to nearest) and the full operator in double-FP32
// arithmetic on FP64 vectors (out = D in, or out = b - D in when b is set); Udf [4][9][V],
// clovdf [2][36][V] with the mass shift
void double_to_df(dfl* dst, const double* src, size_t n, cudaStream_t st);
void fine_dslash_df(cplx<double>* out, const cplx<double>* in, const cplx<double>* b, const cplx<dfl>* Udf,
                    const dfl* clovdf, const Geom& g, int bc_t, int nrhs, size_t rstride, cudaStream_t st);
// per-site inverse of the packed Hermitian 6x6 blocks (LDL^+ in FP64); *err = 1 on a zero pivot
void clover_inverse(double* inv, const double* clov, int V, int* err, cudaStream_t st);
// the Schur SAP tables (either pointer may be null)
void clover_mix(float* mix32, __half2* mixh, const double* clov, const double* inv, const Geom& g, double shift,
                cudaStream_t st);
// FP16 copies: links (no scale, |U_ab| <= 1) and the clover term A - shift (no scale)
void links_to_half(__half2* dst, const cplx<double>* U, size_t n, cudaStream_t st);
void clover_to_half(__half2* dst, const double* A, int V, double shift, cudaStream_t st);
template <typename T>
void links_import(cplx<T>* U, const cplx<double>* gauge_lex, const Geom& g, cudaStream_t st);
template <typename T>
void fine_import(cplx<T>* dst, const cplx<double>* src, const Geom& g, int nrhs, size_t rstride, cudaStream_t st);
template <typename T>
void fine_export(cplx<double>* dst, const cplx<T>* src, const Geom& g, int nrhs, size_t rstride, cudaStream_t st);

// ---- coarse levels --------------------------------------------------------
template <typename T>
void coarse_apply(cplx<T>* out, const cplx<T>* in, const cplx<T>* b, const CoarseOp<T>& op, int nrhs,
                  size_t rstride, int sel, int sel_mu, int in_chir, cudaStream_t st);
// tensor-core coarse stencil on FP16 blocks (whole operator, any batch; see coarse_tc.cu):
// cudaErrorInvalidValue (nothing launched) when the configuration does not fit
cudaError_t coarse_apply_tc(cplx<float>* out, const cplx<float>* in, const cplx<float>* b, const CoarseOp<float>& op,
                            int nrhs, size_t rstride, int ks, cudaStream_t st);
bool coarse_tc_fits(int n, int ks);
size_t coarse_tc_smem(int n, int ks);
// cudaErrorInvalidConfiguration (nothing launched) when a SAP block exceeds what one CTA can hold
template <typename T>
cudaError_t coarse_sap_sweep(cplx<T>* z, const cplx<T>* b, const CoarseOp<T>& op, const int* blocks, int nblocks,
                      int nrhs, size_t rstride, int k_mr, cudaStream_t st);
// all `iters` SAP applications (red then black sweep) in one cooperative launch of clusters that
// stay resident (FP16 blocks, FP32 compute), nbpc (1 or 2) SAP blocks of each colour per cluster;
// *gcnt: a device counter for the launch's barriers.  fits: the smallest nbpc for which all
// clusters are resident at once (*max_clusters: clusters of that shape the device holds, -1: not
// queried)
size_t coarse_sap_persist_smem(const CoarseOp<float>& op, int nbpc);
bool coarse_sap_persist_fits(const CoarseOp<float>& op, int nb0, int nb1, int* max_clusters = nullptr,
                             int* nbpc = nullptr, int min_nbpc = 1);
cudaError_t coarse_sap_persist(cplx<float>* z, const cplx<float>* b, const CoarseOp<float>& op, const int* blocks0,
                               int nb0, const int* blocks1, int nb1, int nrhs, size_t rstride, int k_mr, int iters,
                               int nbpc, unsigned* gcnt, cudaStream_t st);
void coarse_selfinv_build(cplx<double>* inv, const cplx<double>* blk, int V, int n, int* err, cudaStream_t st);
template <typename T>
// prefer: a cluster size (2, 4, 8, 16) to try first, anything else for the default order
int coarse_sap_cluster_plan(const Geom& g, int n, int* CLS_out, int* spc_out, int* nsl_out, int prefer = 0);
// t(A odd) = S^{-1}(a b + c D_oe x)     (even entries of t untouched)
template <typename T>
void coarse_schur_odd(cplx<T>* t, const cplx<T>* x, const cplx<T>* b, const CoarseOp<T>& op, double a, double c,
                      int nrhs, size_t rstride, cudaStream_t st);
// y(A even) = a b + s S x + c D_eo t;  y(A odd) = 0
template <typename T>
void coarse_schur_even(cplx<T>* y, const cplx<T>* x, const cplx<T>* t, const cplx<T>* b, const CoarseOp<T>& op,
                       double a, double s, double c, int nrhs, size_t rstride, cudaStream_t st);
template <typename T>
void coarse_selfinv_apply(cplx<T>* out, const cplx<T>* in, const CoarseOp<T>& op, int parity, int nrhs,
                          size_t rstride, cudaStream_t st);
template <typename T>
void coarse_sub_parity(cplx<T>* y, const cplx<T>* a, const cplx<T>* b, const Geom& g, int n, int parity, int nrhs,
                       size_t rstride, cudaStream_t st);
template <typename T>
void coarse_import(cplx<T>* dst, const cplx<double>* src, const Geom& g, int n, int nrhs, size_t rstride,
                   cudaStream_t st);
template <typename T>
void coarse_export(cplx<double>* dst, const cplx<T>* src, const Geom& g, int n, int nrhs, size_t rstride,
                   cudaStream_t st);
void coarse_blocks_export(cplx<double>* dst, const cplx<double>* blk, const Geom& g, int n, cudaStream_t st);
// FP16 copy of the blocks with one scale per site: s = max |re|, |im| over the site's 9 blocks
void blocks_to_half(__half2* dst, float* scale, const cplx<double>* blk, int V, int n, cudaStream_t st);

// ---- coarsest level: cluster-resident odd-even GMRES ---------------------------
struct CoarsestPlanIn {
  int n_even, n_odd, n, m;
};
struct CoarsestPlan {
  int CL = 0, nep = 0, nop = 0, threads = 0;
  size_t smem = 0;
  int res_nr = 0;        // > 0: the resident variant (FP32 on FP16 blocks) fits
  size_t res_smem = 0;
};
struct CoarsestGeo {
  const int* even = nullptr;
  const int* odd = nullptr;
  const int* nbr_e_of_o = nullptr;   // [n_odd][8]
  const int* nbr_o_of_e = nullptr;   // [n_even][8]
  int n_even = 0, n_odd = 0;
};
template <typename T>
int coarsest_cluster_plan(const CoarsestPlanIn& in, CoarsestPlan* plan);
template <typename T>
cudaError_t coarsest_cluster_solve(cplx<T>* x, const cplx<T>* b, const CoarseOp<T>& op, const CoarsestPlan& plan,
                            const CoarsestGeo& geo, int nrhs, size_t rstride, int m, int max_cycles, double tol,
                            int* iters, cudaStream_t st);

// ---- transfer ---------------------------------------------------------------
// out(A)[s*N + j] = sum_{x in A, f in s} conj(P_j(x, f)) in(x, f)
// (Ph, pscale): optional FP16 copy of P with per-(aggregate, chirality) scales (FP32 compute only)
// tc_ks >= 1 (FP32 compute on FP16 P only): the tensor-core kernel with that k-split, P read once
// per batch (transfer_tc.cu)
template <typename T>
void restrict_op(cplx<T>* out, const cplx<T>* in, const cplx<T>* P, const Geom& gf, const Geom& gc, bool fine,
                 int n, int N, int nrhs, size_t in_rstride, size_t out_rstride, size_t out_site_stride,
                 cudaStream_t st, const __half2* Ph = nullptr, const float* pscale = nullptr, int tc_ks = 0);
// out(x, f) = [out +] sum_j P_j(x, f) in(A(x))[s(f)*N + j]
// batch != 0 (FP32 compute on FP16 P only): one CTA per aggregate for the whole batch (P read once)
template <typename T>
void prolong_op(cplx<T>* out, const cplx<T>* in, const cplx<T>* P, const Geom& gf, const Geom& gc, bool fine, int n,
                int N, int nrhs, size_t out_rstride, size_t in_rstride, bool accumulate, cudaStream_t st,
                const __half2* Ph = nullptr, const float* pscale = nullptr, int batch = 0);
cudaError_t restrict_tc(cplx<float>* out, const cplx<float>* in, const __half2* Ph, const float* pscale,
                        const Geom& gf, const Geom& gc, bool fine, int n, int N, int nrhs, size_t in_rstride,
                        size_t out_rstride, size_t out_site_stride, int ks, cudaStream_t st);
bool restrict_tc_fits(int N, int ks);
cudaError_t prolong_batch(cplx<float>* out, const cplx<float>* in, const __half2* Ph, const float* pscale,
                          const Geom& gf, const Geom& gc, bool fine, int n, int N, int nrhs, size_t out_rstride,
                          size_t in_rstride, bool accumulate, cudaStream_t st);
void p_to_half(__half2* Ph, float* pscale, const cplx<double>* P, const Geom& g, bool fine, int n, int N,
               cudaStream_t st);
// in-place CGS2 per aggregate and chirality of N fields (FP64); err set on rank deficiency
void orthonormalise(cplx<double>* P, const Geom& g, bool fine, int n, int N, int* err, cudaStream_t st);

// ---- random fields (setup) -----------------------------------------------------
// nfields complex N(0,1) fields j0 .. j0+nfields-1 of `level` in that level's layout
// (fine: [12][V], coarse: [V][n]), rstride complex elements apart: Philox4x32-10 on the
// counter (lexicographic site, dof, field, level) under the 64-bit seed, then Box-Muller
void draw_fields(cplx<double>* dst, const Geom& g, bool fine, int n, int nfields, int j0, int level, uint64_t seed,
                 size_t rstride, cudaStream_t st);

// ---- BLAS-1 (batched over rhs, rstride complex elements between rhs) ----------
template <typename T>
void blas_dot(cplx<double>* res, const cplx<T>* x, const cplx<T>* y, size_t len, int nrhs, size_t rstride,
              cudaStream_t st);
template <typename T>
void blas_norm2(double* res, const cplx<T>* x, size_t len, int nrhs, size_t rstride, cudaStream_t st);
// res[rhs*res_stride + i] = V_i^+ w, V_i at V + i*vstride + rhs*rstride
template <typename T>
void blas_multidot(cplx<double>* res, int res_stride, const cplx<T>* V, size_t vstride, int m, const cplx<T>* w,
                   size_t len, int nrhs, size_t rstride, cudaStream_t st);
void reserve_partials(int nrhs, int m, cudaStream_t st);   // per stream
// a[i] = 1 / a[i] (0 where a[i] = 0)
void blas_recip(double* a, int n, cudaStream_t st);
// y += sign * sum_i c[rhs*cstride + i] V_i
template <typename T>
void blas_multiaxpy(cplx<T>* y, const cplx<T>* V, size_t vstride, int m, const cplx<double>* c, int cstride,
                    double sign, size_t len, int nrhs, size_t rstride, cudaStream_t st);
// the same two operations in double-FP32 arithmetic on FP64 vectors (outer Gram-Schmidt option)
void blas_multidot_df(cplx<double>* res, int res_stride, const cplx<double>* V, size_t vstride, int m,
                      const cplx<double>* w, size_t len, int nrhs, size_t rstride, cudaStream_t st);
void blas_multiaxpy_df(cplx<double>* y, const cplx<double>* V, size_t vstride, int m, const cplx<double>* c,
                       int cstride, double sign, size_t len, int nrhs, size_t rstride, cudaStream_t st);
// y = a[rhs] * x   (a real, from device memory)
template <typename T>
void blas_scale_to(cplx<T>* y, const cplx<T>* x, const double* a, size_t len, int nrhs, size_t rstride,
                   cudaStream_t st);
template <typename T>
void blas_axpy(cplx<T>* y, const cplx<T>* x, double a, size_t len, int nrhs, size_t rstride, cudaStream_t st);
template <typename To, typename Ti>
void blas_convert(cplx<To>* y, const cplx<Ti>* x, size_t len, int nrhs, size_t ystride, size_t xstride,
                  cudaStream_t st);
template <typename T>
void blas_zero(cplx<T>* y, size_t len, int nrhs, size_t rstride, cudaStream_t st);
template <typename T>
void real_convert(T* y, const double* x, size_t len, cudaStream_t st);

// ---- GMRES bookkeeping (per rhs, FP64 scalars) ---------------------------------
struct GmresState {
  cplx<double>* H;      // [rhs][m+1][m] Hessenberg, rotated to R in place
  double* cs;           // [rhs][m]
  cplx<double>* sn;     // [rhs][m]
  cplx<double>* g;      // [rhs][m+1]
  cplx<double>* h1;     // [rhs][m+1] first CGS pass coefficients
  cplx<double>* h2;     // [rhs][m+1] second CGS pass
  double* wnorm;        // [rhs]
  double* inv;          // [rhs] 1 / ||w||
  double* beta;         // [rhs] initial residual norm of the cycle
  double* target;       // [rhs] absolute stopping threshold
  double* est;          // [rhs] |g_{j+1}|
  int* done;            // [rhs] stopped in this cycle
  int* kr;              // [rhs] iterations taken in this cycle
  cplx<double>* y;      // [rhs][m]
  int* conv;            // [rhs] converged (device-driven solver)
  int* iters;           // [rhs] iterations over all cycles (device-driven solver)
  double* bnorm;        // [rhs] ||b||
  int* ctl;             // [4]: j, cycle, arrival counter
  int m;
};
void gmres_begin(const GmresState& s, int nrhs, cudaStream_t st);                // g = beta e1, inv = 1/beta
void gmres_step(const GmresState& s, int j, int nrhs, cudaStream_t st);          // rotations, new g, done flags
void gmres_solve_y(const GmresState& s, int nrhs, cudaStream_t st);              // y = R^{-1} g (k_r per rhs)

// device-driven variant (graph capture with conditional WHILE nodes)
void kry_start(const GmresState& s, int nrhs, double tol, cudaGraphConditionalHandle hcycle, cudaStream_t st);
template <typename T>
void kry_cycle_begin(const GmresState& s, cplx<T>* V0, cplx<T>* cur, const cplx<T>* r, size_t vlen, int nrhs,
                     cudaGraphConditionalHandle hinner, cudaStream_t st);
template <typename T>
cudaError_t kry_arnoldi(const GmresState& s, cplx<T>* V, size_t vstride, cplx<T>* Z, const cplx<T>* zcur, cplx<T>* w,
                        cplx<T>* cur, size_t vlen, int nrhs, cudaGraphConditionalHandle hinner, cudaStream_t st);
// queries (once, outside any stream capture) the cluster size the split Arnoldi step can use
void kry_prepare();
void kry_cycle_end(const GmresState& s, int nrhs, int max_cycles, cudaGraphConditionalHandle hcycle, cudaStream_t st);

}  // namespace dd
