// ok_kernels.h -- kernel launchers shared between the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include "ok_internal.cuh"

namespace okg {

// Scalars of the residual / projection kernels (see ok_fem.cu).
struct ResidualCoefs {
  double a11;    // 1 + dt theta sigma
  double bn;     // 1 - dt (1 - theta) sigma
  double dsm;    // dt sigma m
  double dth;    // dt theta
  double dth1;   // dt (1 - theta)
  double hd;     // h^d       (mass scale)
  double hk;     // h^(d-2)   (stiffness scale)
  double eps2;   // eps^2
  double vol;    // |T| = h^d / d!
  double a4;     // d! / (d+4)!
  double a2;     // d! / (d+2)!
  double msum4;  // 2D: row sum of the reference mass table of an interior vertex
};

// y = alpha J z + beta y0 (y0 may be null: y = J z)
struct JCoefs {
  double a11hd;  // (1 + dt theta sigma) h^d
  double dthhk;  // dt theta h^(d-2)
  double hd;
  double alpha, beta;
};

void launch_residual(int dim, const Geom& g, const double* WM, const double* WK, const ResidualCoefs& rc,
                     const double* un, const double* wn, const double* u, const double* w, double* f,
                     cudaStream_t s);
void launch_initw_rhs(int dim, const Geom& g, const double* WK, const ResidualCoefs& rc, const double* u,
                      double* out, cudaStream_t s);
// e[v] = eps^2/2 u_v (K u)_v, e[N_v + v] = vertex share of 1/4 int (1 - u_h^2)^2 (2 N_v values)
void launch_energy_local(int dim, const Geom& g, const double* WK, const ResidualCoefs& rc, const double* u,
                         double* e, cudaStream_t s);
void launch_assemble_c(int dim, const Geom& g, const ResidualCoefs& rc, const double* u, double* coef,
                       float* coef32, cudaStream_t s);
template <typename TZ>
void launch_apply_j(int dim, const Geom& g, const double* WM, const double* WK, const JCoefs& jc,
                    const double* coef, const TZ* z, double* y, const double* y0, cudaStream_t s);
template <typename T, typename TV>
void launch_cstep(int dim, const Geom& g, const T* coef, const TV* v2, T vscale, const T* y1, T yscale, T* t,
                  cudaStream_t s);
// batched forms (same grid size, `count` <= BATCH_MAX problems; the reference
// tables WM, WK are the same for every problem of a grid size)
template <typename TZ> struct ApplyJItem {
  JCoefs jc;
  const double* coef;
  const TZ* z;
  double* y;
};
template <typename TZ>
void launch_apply_j_b(int dim, const Geom& g, const double* WM, const double* WK, const ApplyJItem<TZ>* items,
                      int count, cudaStream_t s);
template <typename T, typename TV> struct CStepItem {
  const T* coef;
  const TV* v2;
  T vscale;
  const T* y1;
  T yscale;
  T* t;
};
template <typename T, typename TV>
void launch_cstep_b(int dim, const Geom& g, const CStepItem<T, TV>* items, int count, cudaStream_t s);
template <typename T>
void launch_schur_resid(int dim, const Geom& g, const T* WM, T hd, const T* coef, const T* t, const T* y,
                        const T* a, T ascale, T* out, cudaStream_t s);

// ---- Chebyshev / multigrid (ok_mg.cu) ------------------------------------
// All operate on one level with a per-class weight table W (already scaled
// to the level) and per-class inverse diagonal dinv.
// r = s*b, d = dinv r / th                          (x = 0 start)
template <typename T, typename TB>
void launch_cheb_init(int dim, const Geom& g, const T* dinv, const TB* b, T bscale, T* r, T* d, T inv_th,
                      cudaStream_t s);
// r = b - W x, d = dinv r / th
template <typename T>
void launch_resid_init(int dim, const Geom& g, const T* W, const T* dinv, const T* b, const T* x, T* r, T* d,
                       T inv_th, cudaStream_t s);
// x = (first ? 0 : x) + d_in; r -= W d_in; d_out = c1 d_in + c2 dinv r
template <typename T>
void launch_cheb_step(int dim, const Geom& g, const T* W, const T* dinv, T* x, T* r, const T* d_in, T* d_out,
                      T c1, T c2, bool first, cudaStream_t s);
// x = (first ? 0 : x) + d_in; if (r) r -= W d_in; if (out) out = oscale * x
template <typename T, typename TO>
void launch_cheb_last(int dim, const Geom& g, const T* W, T* x, T* r, const T* d_in, bool first, TO* out,
                      T oscale, cudaStream_t s);
// b_c = P^T r_f; with dinv also r = b_c, d = dinv b_c inv_th on the coarse
// level (launch_cheb_init from zero, folded into the same launch)
template <typename T>
void launch_restrict(int dim, const Geom& gf, const Geom& gc, const T* rf, T* bc, cudaStream_t s,
                     const T* dinv = nullptr, T* r = nullptr, T* d = nullptr, T inv_th = (T)0);
// x_f += P x_c (with dc: x_f += P (x_c + d_c), the coarse level's last
// smoothing step x_c += d_c folded in)
template <typename T>
void launch_prolong_add(int dim, const Geom& gf, const Geom& gc, T* xf, const T* xc, cudaStream_t s,
                        const T* dc = nullptr);
// x = Ainv b on the coarsest level (dense, row stride nc), one thread block
template <typename T>
void launch_coarse_solve(long long nc, const T* Ainv, const T* b, T* x, cudaStream_t s);
// the same by many blocks; Ainv has row stride ld = gemv_ld(nc) and zero padding
long long gemv_ld(long long nc, size_t elem);
template <typename T>
void launch_coarse_gemv(long long nc, long long ld, const T* Ainv, const T* b, T* x, cudaStream_t s);
template <typename T>
cudaError_t prepare_coarse_gemv(long long nc);
// y = alpha W x (+ beta y0 when y0 != null), first NO offsets: full (M-like) or axis (K)
template <typename T, typename TX, typename TY>
void launch_op_apply(int dim, const Geom& g, const T* W, bool axis_only, const TX* x, TY* y, T alpha,
                     const TY* y0, T beta, cudaStream_t s);
// ---- 3D steps by z-marching blocks (ok_plane3.cu) -------------------------
// The same operations as launch_resid_init / launch_cheb_step /
// launch_cheb_last (with r) / launch_op_apply on a 3D level, bitwise equal;
// each value of the stencil vector is read once per block (plane ring in
// shared memory).
// `shape` selects the block shape (0..PLANE_SHAPES-1: 32x8 columns x 16
// planes, 32x4 x 32, 64x4 x 16, 32x8 x 32).
constexpr int PLANE_SHAPES = 4;
enum PlaneMode { PM_RESID = 0, PM_STEP = 1, PM_LAST = 2, PM_OP = 3 };
template <typename T, typename TS, typename TO> struct PlaneArgs {
  Geom g;
  const T* W;          // class table of the operator (level-scaled)
  const T* dinv;       // 1 / diagonal per class (RESID, STEP)
  const TS* s;         // the vector the stencil reads: x (RESID, OP) or d (STEP, LAST)
  T* x;                // STEP, LAST: iterate (in-out)
  T* r;                // RESID: out; STEP, LAST: in-out
  T* d;                // RESID: d out; STEP: d_out
  const T* b;          // RESID: right-hand side
  TO* out;             // LAST: optional cast of x; OP: y
  const TO* y0;        // OP: optional y0
  T c1, c2, inv_th, oscale, alpha, beta;
  int first;           // STEP, LAST: x starts from zero
  int axis_only;       // OP: first 2d + 1 offsets (K-like tables)
};
// batched form: one launch of `mode` for `count` <= BATCH_MAX problems on grids of one size
template <typename T, typename TS, typename TO>
void launch_plane3_b(int mode, const PlaneArgs<T, TS, TO>* items, int count, int shape, cudaStream_t s);
template <typename T>
void launch_resid_init3(const Geom& g, const T* W, const T* dinv, const T* b, const T* x, T* r, T* d, T inv_th,
                        cudaStream_t s, int shape);
template <typename T>
void launch_cheb_step3(const Geom& g, const T* W, const T* dinv, T* x, T* r, const T* d_in, T* d_out, T c1, T c2,
                       bool first, cudaStream_t s, int shape);
template <typename T, typename TO>
void launch_cheb_last3(const Geom& g, const T* W, T* x, T* r, const T* d_in, bool first, TO* out, T oscale,
                       cudaStream_t s, int shape);
template <typename T, typename TX, typename TY>
void launch_op_apply3(const Geom& g, const T* W, bool axis_only, const TX* x, TY* y, T alpha, const TY* y0, T beta,
                      cudaStream_t s, int shape);

// Fused coarse V-cycle: levels Lc..L of the hierarchy in one thread block with
// every level vector in shared memory (x, b, r, d0, d1 at off[l]).
constexpr int COARSE_MAXLEV = 8;
constexpr size_t COARSE_SMEM_MAX = 200 * 1024;   // shared-memory budget of the fused coarse V-cycle
constexpr long long COARSE_NC_MAX = 4913;         // largest coarsest level solved densely
template <typename T> struct CoarseArgs {
  int nlev;                          // levels in the fused part (>= 2)
  Geom g[COARSE_MAXLEV];
  const T* W[COARSE_MAXLEV];         // S_hat weight tables (global)
  const T* dinv[COARSE_MAXLEV];
  long long off[COARSE_MAXLEV];      // element offset of the level's 5 vectors
  long long toff[COARSE_MAXLEV];     // element offset of the level's W and dinv copies
  unsigned mul[COARSE_MAXLEV];       // ceil(2^32 / (n+1)): i / (n+1) = umulhi(i, mul)
  unsigned mulI[COARSE_MAXLEV];      // ceil(2^32 / (n-1)) for the interior vertices (n > 2)
  const T* Ainv;                     // coarsest dense inverse (global)
  T inv_th;                          // smoother 1/centre
  T c1[16], c2[16];                  // smoother coefficients per step
  int nu_pre, nu_post;
};
// b_in: right-hand side of level Lc; x_in: start iterate (null = zero); x_out: result
template <typename T>
void launch_coarse_vcycle(int dim, const CoarseArgs<T>& a, size_t smem, const T* b_in, const T* x_in, T* x_out,
                          cudaStream_t s);
// allow the fused kernel its dynamic shared memory (call before capture).  The
// limit is a property of the kernel shared by every handle in the process, so
// it is always set to the largest any handle uses (COARSE_SMEM_MAX), never to
// one handle's need.
template <typename T>
cudaError_t prepare_coarse_vcycle(int dim, size_t smem);

// ---- register-strip tile kernels, 2D (ok_tile.cu) ------------------------
// compiled window shapes of the strip kernels (columns x rows, rows per
// thread): float 0: 32 x 32 by 2, 1: 64 x 32 by 8, 2: 64 x 32 by 4,
// 3: 64 x 64 by 4, 4: 128 x 32 by 4; float64 0: 32 x 16 by 2, 1: 64 x 32 by
// 2, 2: 64 x 32 by 4, 3: 32 x 32 by 4, 4: 64 x 16 by 2
constexpr int STRIP_SHAPES = 5;
template <typename T> struct TileSmooth {
  Geom g, gc;             // this level and the next coarser one
  const T* W;             // S_hat table of this level
  const T* dinv;
  const T* WM;            // M table of this level (post kernel's optional M x)
  T inv_th, c1, c2;       // smoother: 1/centre, coefficients of the middle step
  int tile;               // window shape (0 .. STRIP_SHAPES-1)
};
template <typename T> struct TileMass {
  Geom g;
  const T* WM;            // M table (finest level)
  const T* dinvM;
  const T* coef;          // C = -eps^2 K - M_E coefficients, symmetric store
  int q;                  // Chebyshev steps (halo width), 1..16
  T inv_th, inv_a11;
  T c1[16], c2[16];
  T *sx, *sr, *sd;        // x, r, d handed from the first launch to the second (N_v each)
};
// pre-smoothing (2 steps from x_in, or zero when x_in is null), restriction into bc
template <typename T>
void launch_tile_pre(const TileSmooth<T>& a, const T* x_in, const T* b, T* x_out, T* bc, cudaStream_t s);
// x_out = post-smoothed (x_in + P xc); mx_out = M x_out (optional); out = oscale x_out (optional)
template <typename T, typename TO>
void launch_tile_post(const TileSmooth<T>& a, const T* x_in, const T* xc, const T* b, T* x_out, T* mx_out, TO* out,
                      T oscale, cudaStream_t s);
// z1 = A~^{-1} v1, t_out = v2 - C z1
template <typename T, typename TZ>
void launch_tile_amass(const TileMass<T>& a, const double* v, TZ* z1, T* t_out, cudaStream_t s);
template <typename T>
cudaError_t prepare_tiles(int q);
// batched forms: one launch for `count` <= BATCH_MAX problems of the same grid
// and window width (items[i] carries problem i's arguments; blockIdx.z = i)
template <typename T> struct StripPreItem {
  TileSmooth<T> a;
  const T* x_in;
  const T* b;
  T* x_out;
  T* bc;
};
template <typename T, typename TO> struct StripPostItem {
  TileSmooth<T> a;
  const T *x_in, *xc, *b;
  T *x_out, *mx_out;
  TO* out;
  T oscale;
};
template <typename T, typename TZ> struct AmassItem {
  TileMass<T> a;
  const double* v;
  TZ* z1;
  T* t_out;
};
template <typename T>
void launch_tile_pre_b(const StripPreItem<T>* items, int count, cudaStream_t s);
template <typename T, typename TO>
void launch_tile_post_b(const StripPostItem<T, TO>* items, int count, cudaStream_t s);
template <typename T, typename TZ>
void launch_tile_amass_b(const AmassItem<T, TZ>* items, int count, cudaStream_t s);
// thread blocks of a pre-smoothing launch on level g with window width `tile`
template <typename T>
long long strip_blocks(const Geom& g, int tile);

// The bottom of a 2D V-cycle in one launch of one thread-block cluster: the
// pre-smoothing kernels' work on levels 0..nl-1 of the argument (finest
// first), the dense solve of the coarsest level, then the post-smoothing
// kernels' work back up, phases separated by cluster barriers.  Level i
// pre-smooths from zero on rhs[i] into P[i] and restricts into rhs[i+1];
// rhs[nl] is the coarsest level's right-hand side, xc its solution; level i
// post-smooths P[i] + prolongated (i == nl-1 ? xc : Q[i+1]) into Q[i].
constexpr int LOW_MAXLEV = 6;
template <typename T> struct LowArgs {
  int nl;
  TileSmooth<T> ts[LOW_MAXLEV];
  T* P[LOW_MAXLEV];
  T* Q[LOW_MAXLEV];
  T* rhs[LOW_MAXLEV + 1];
  long long nc, ldA;       // coarsest level: unknowns, padded row stride of its inverse
  const T* A;              // zero-padded dense inverse
  T* xc;
};
// cluster size usable for the kernel on this device (16, 8, or 0: none); sets
// the kernel's attributes for a coarsest level of nc unknowns
template <typename T>
int prepare_low_vcycle(long long nc);
template <typename T>
void launch_low_vcycle(const LowArgs<T>& a, int cluster, cudaStream_t s);

// ---- batched multigrid steps (one launch for `count` <= BATCH_MAX problems
// on grids of the same size; items[i] carries problem i's arguments) --------
template <typename T, typename TB> struct ChebInitItem {
  const T* dinv;
  const TB* b;
  T bscale;
  T* r;
  T* d;
  T inv_th;
};
template <typename T, typename TO> struct ChebLastItem {
  const T* W;
  T *x, *r;
  const T* din;
  int first;
  TO* out;
  T oscale;
};
template <typename T> struct TransferItem {
  T* fine;          // restrict: fine residual (read); prolong: fine iterate (updated)
  T* coarse;        // restrict: coarse right-hand side (written); prolong: coarse correction (read)
  const T* dinv;    // restrict, optional: also start the coarse smoothing from zero (r, d below)
  T* r;
  T* d;
  T inv_th;
  const T* dc;      // prolong, optional: the coarse level's last step folded in (P (coarse + dc))
};
template <typename T> struct GemvItem {
  const T* A;
  const T* b;
  T* x;
};
template <typename T> struct CoarseVItem {
  const CoarseArgs<T>* a;   // device copy of the problem's CoarseArgs
  const T* b_in;
  const T* x_in;
  T* x_out;
};
template <typename T, typename TB>
void launch_cheb_init_b(int dim, const Geom& g, const ChebInitItem<T, TB>* items, int count, cudaStream_t s);
template <typename T, typename TO>
void launch_cheb_last_b(int dim, const Geom& g, const ChebLastItem<T, TO>* items, int count, cudaStream_t s);
template <typename T>
void launch_restrict_b(int dim, const Geom& gf, const Geom& gc, const TransferItem<T>* items, int count,
                       cudaStream_t s);
template <typename T>
void launch_prolong_add_b(int dim, const Geom& gf, const Geom& gc, const TransferItem<T>* items, int count,
                          cudaStream_t s);
// the coarsest solve x = A^{-1} b: many-block GEMV (gemv, padded stride ld) or one block per problem
template <typename T>
void launch_coarse_solve_b(long long nc, long long ld, bool gemv, const GemvItem<T>* items, int count,
                           cudaStream_t s);
template <typename T>
void launch_coarse_vcycle_b(int dim, const CoarseVItem<T>* items, int count, size_t smem, cudaStream_t s);

// dense matrix of a level operator (row-major nv x nv) from its class table
void launch_dense_from_table(int dim, const Geom& g, const double* W, double* A, cudaStream_t s);
// in-place Gauss--Jordan inverse of an SPD matrix (single block); work: n x 2n
void launch_gauss_jordan(long long n, const double* A, double* work, double* Ainv, cudaStream_t s);

// ---- Krylov (ok_krylov.cu) -----------------------------------------------
struct KrylovState;   // device-resident Arnoldi/Givens state (ok_krylov.cu)
struct RedScratch {
  double* partials;    // RED_MAX_BLOCKS * KRYLOV_MAX
  unsigned int* counter;
};
int krylov_blocks();
// ks->h1[0..K) = V^T w       (V: K vectors with leading dimension ldv)
// (skip: device flag, the launches return at once when it is set; nw0: also ||w||^2 there)
void launch_multidot(const double* V, long long ldv, int K, const double* w, long long N, RedScratch rs,
                     double* out, cudaStream_t s, const int* skip = nullptr, double* nw0 = nullptr);
// w -= V h_in; h_out = V^T w
void launch_update_multidot(const double* V, long long ldv, int K, const double* h_in, double* w, long long N,
                            RedScratch rs, double* h_out, cudaStream_t s);
// w -= V h2; then Arnoldi column j finalisation (h1 + h2) + Givens in the last block
void launch_update_norm_givens(const double* V, long long ldv, int K, double* w, long long N, RedScratch rs,
                               KrylovState* ks, int j, cudaStream_t s, const int* skip = nullptr);
// w -= V h1; ||w||^2 against ks->nw0 decides the second pass (sets ks->skip2;
// `single`: never); without it the column (h1) and its Givens rotation are
// finished here
void launch_update_norm_check(const double* V, long long ldv, int K, double* w, long long N, RedScratch rs,
                              KrylovState* ks, int j, cudaStream_t s, bool single = false);
// w *= ks->inv_eta
void launch_scale_by(double* w, long long N, const double* factor, cudaStream_t s);
// one problem of a batched Arnoldi orthogonalisation
struct KrylovItem {
  const double* V;       // basis v_0..v_j, leading dimension ldv
  long long ldv;
  double* w;             // the vector being orthogonalised (becomes v_{j+1})
  long long N;
  double* partials;      // the problem's reduction scratch
  unsigned int* counter;
  KrylovState* ks;
  int h_out_is_h2;       // internal: multidot result into h2 instead of h1
};
// CGS2 orthogonalisation of step j for `count` <= BATCH_MAX problems per launch
void launch_cgs2_batch(const KrylovItem* items, int count, int K, int j, cudaStream_t s);
// out = ||x||_2 (device scalar)
void launch_norm(const double* x, long long N, RedScratch rs, double* out, cudaStream_t s);
// cycle start: v0 = r / beta with beta = ||r|| on device; ks reset
void launch_cycle_start(KrylovState* ks, const double* beta, double thresh, cudaStream_t s);
// k_cond_set(cudaGraphConditionalHandle, const KrylovState*): sets a graph's IF
// condition from the cycle's continue flag
void* cond_set_kernel();
// y = H^{-1} g (upper triangular, size k)
void launch_lsq(KrylovState* ks, int k, cudaStream_t s);
// x += sum_k y_k Z_k
template <typename TZ>
void launch_multi_axpy(const TZ* Z, long long ldz, int K, const KrylovState* ks, double* x, long long N,
                       cudaStream_t s);
// y = a x + b y, typed
template <typename TX, typename TY>
void launch_axpby(long long N, double a, const TX* x, double b, TY* y, cudaStream_t s);
// flag |= any non-finite in x
void launch_check_finite(const double* x, long long N, int* flag, cudaStream_t s);
size_t krylov_state_bytes();
// sets the message ok_last_error() returns (defined in ok_api.cu)
void set_last_error(const char* msg);
double* ks_resid_ptr(KrylovState* ks);
double* ks_eta_ptr(KrylovState* ks);
double* ks_beta_ptr(KrylovState* ks);
double* ks_h1_ptr(KrylovState* ks);
double* ks_h2_ptr(KrylovState* ks);
double* ks_nw0_ptr(KrylovState* ks);
int* ks_skip2_ptr(KrylovState* ks);
int* ks_passes2_ptr(KrylovState* ks);
// the Arnoldi matrix of the current cycle, reduced by its Givens rotations
// (column j at H + (KRYLOV_MAX + 1) j), the rotations and the steps taken
const double* ks_H_ptr(const KrylovState* ks);
const double* ks_cs_ptr(const KrylovState* ks);
const double* ks_sn_ptr(const KrylovState* ks);
const double* ks_nsteps_ptr(const KrylovState* ks);

}  // namespace okg
