// ok_mg.cu -- Chebyshev--Jacobi iterations and geometric multigrid transfers.
//
// Chebyshev semi-iteration (Golub & Varga 1961) for W x = b with the Jacobi
// preconditioner D = diag(W) on an eigenvalue interval [lo, hi] of D^{-1} W,
// centre th, half-width de, in the three-term form
//     r_0 = b - W x_0,  d_0 = D^{-1} r_0 / th
//     x_{k+1} = x_k + d_k,   r_{k+1} = r_k - W d_k,
//     d_{k+1} = c1_k d_k + c2_k D^{-1} r_{k+1}
// (c1_k = rho_{k+1} rho_k, c2_k = 2 rho_{k+1}/de, rho_0 = de/th,
//  rho_{k+1} = 1/(2 th/de - rho_k), computed on the host).
// Used for A~^{-1} = (Chebyshev on M)/(1 + dt theta sigma) (Sec. 3: A is a
// scaled mass matrix) and as the smoother of the V-cycles for
// S_hat = M + eps sqrt(c) K.
//
// Transfers between nested uniform meshes (n_f = 2 n_c): the fine vertex 2i+b,
// b in {0,1}^d, is the midpoint of the coarse edge (i, i+b), so
//     (P x_c)(2i+b) = (x_c(i) + x_c(i+b)) / 2,     (P x_c)(2i) = x_c(i),
//     (P^T r_f)(i)  = r_f(2i) + 1/2 sum_{b != 0} [r_f(2i+b) + r_f(2i-b)],
// the second sum running over the same offsets +-b as the P1 stencil.
#include <algorithm>

#include "ok_internal.cuh"
#include "ok_kernels.h"
#include "ok_stencil.cuh"

namespace okg {

static constexpr int BX = 128;

static inline dim3 grid_of(int dim, const Geom& g) {
  return dim3((unsigned)(((long long)g.n1 * g.n1 + BX - 1) / BX), 1, dim == 3 ? g.n1 : 1);
}

// ---------------------------------------------------------------------------
// one kernel per step
// ---------------------------------------------------------------------------
// The level's class tables (fixed at setup) are copied into shared memory
// before the wait on the previous kernel; every vertex then reads its weights
// there instead of from global memory.
template <int D, typename T>
__device__ __forceinline__ void stage_level(T* sW, T* sD, const T* __restrict__ W, const T* __restrict__ dinv) {
  constexpr int NT = Topo<D>::NCLASS * Topo<D>::NOFF;
  pdl_launch_dependents();
  if (W)
    for (int i = threadIdx.x; i < NT; i += blockDim.x) sW[i] = W[i];
  if (dinv)
    for (int i = threadIdx.x; i < Topo<D>::NCLASS; i += blockDim.x) sD[i] = dinv[i];
  __syncthreads();
  pdl_wait();
}
#define OK_LEVEL_SMEM(D, T)                                  \
  __shared__ T sW[Topo<D>::NCLASS * Topo<D>::NOFF];          \
  __shared__ T sD[Topo<D>::NCLASS]
template <int D, typename T, typename TB>
__global__ void __launch_bounds__(BX) k_cheb_init(Geom g, const T* __restrict__ dinv, const TB* __restrict__ b,
                                                  T bscale, T* __restrict__ r, T* __restrict__ d, T inv_th) {
  OK_LEVEL_SMEM(D, T);
  stage_level<D, T>(sW, sD, (const T*)nullptr, dinv);
  Vtx<D> v;
  if (!vertex_of_thread<D>(g, v)) return;
  cheb_init_at<D, T, TB>(v, sD, b, bscale, r, d, inv_th);
}

template <int D, typename T>
__global__ void __launch_bounds__(BX) k_resid_init(Geom g, const T* __restrict__ W, const T* __restrict__ dinv,
                                                   const T* __restrict__ b, const T* __restrict__ x,
                                                   T* __restrict__ r, T* __restrict__ d, T inv_th) {
  OK_LEVEL_SMEM(D, T);
  stage_level<D, T>(sW, sD, W, dinv);
  Vtx<D> v;
  if (!vertex_of_thread<D>(g, v)) return;
  resid_init_at<D, T>(g, v, sW, sD, b, x, r, d, inv_th);
}

template <int D, typename T>
__global__ void __launch_bounds__(BX) k_cheb_step(Geom g, const T* __restrict__ W, const T* __restrict__ dinv,
                                                  T* __restrict__ x, T* __restrict__ r, const T* __restrict__ din,
                                                  T* __restrict__ dout, T c1, T c2, int first) {
  OK_LEVEL_SMEM(D, T);
  stage_level<D, T>(sW, sD, W, dinv);
  Vtx<D> v;
  if (!vertex_of_thread<D>(g, v)) return;
  cheb_step_at<D, T>(g, v, sW, sD, x, r, din, dout, c1, c2, first != 0);
}

template <int D, typename T, typename TO>
__global__ void __launch_bounds__(BX) k_cheb_last(Geom g, const T* __restrict__ W, T* __restrict__ x,
                                                  T* __restrict__ r, const T* __restrict__ din, int first,
                                                  TO* __restrict__ out, T oscale) {
  OK_LEVEL_SMEM(D, T);
  stage_level<D, T>(sW, sD, r ? W : (const T*)nullptr, (const T*)nullptr);
  Vtx<D> v;
  if (!vertex_of_thread<D>(g, v)) return;
  cheb_last_at<D, T, TO>(g, v, sW, x, r, din, first != 0, out, oscale);
}

// restriction bc = P^T rf; with dinv, also the coarse level's first
// smoothing start from zero (cheb_init_at on bc: r = bc, d = D^{-1} bc / th),
// which would otherwise be the next launch
template <int D, typename T>
__global__ void __launch_bounds__(BX) k_restrict(Geom gf, Geom gc, const T* __restrict__ rf, T* bc,
                                                 const T* __restrict__ dinv, T* __restrict__ r, T* __restrict__ d,
                                                 T inv_th) {
  OK_LEVEL_SMEM(D, T);
  stage_level<D, T>(sW, sD, (const T*)nullptr, dinv);
  Vtx<D> v;                               // coarse vertex
  if (!vertex_of_thread<D>(gc, v)) return;
  restrict_at<D, T>(gf, v, rf, bc);
  if (dinv) cheb_init_at<D, T, T>(v, sD, bc, (T)1, r, d, inv_th);
}

// prolongation xf += P xc (with dc: P (xc + dc), see prolong_add_at)
template <int D, typename T>
__global__ void __launch_bounds__(BX) k_prolong_add(Geom gf, Geom gc, T* __restrict__ xf, const T* __restrict__ xc,
                                                    const T* __restrict__ dc) {
  pdl_entry();
  Vtx<D> v;                               // fine vertex
  if (!vertex_of_thread<D>(gf, v)) return;
  prolong_add_at<D, T>(gc, v, xf, xc, dc);
}

// one block; warp per row
template <typename T>
__global__ void __launch_bounds__(512) k_coarse_solve(long long nc, const T* __restrict__ A, const T* __restrict__ b,
                                                      T* __restrict__ x) {
  pdl_entry();
  coarse_rows<T>(nc, A, b, x, threadIdx.x >> 5, blockDim.x >> 5);
}

// ---- batched forms (grid z folds the problem index, see batch_problem) -----
template <int D, typename T, typename TB>
__global__ void __launch_bounds__(BX) k_cheb_init_b(Batch<ChebInitItem<T, TB>> B, Geom g) {
  OK_LEVEL_SMEM(D, T);
  const ChebInitItem<T, TB>& a = B.a[batch_problem<D>(g)];
  stage_level<D, T>(sW, sD, (const T*)nullptr, a.dinv);
  Vtx<D> v;
  if (!vertex_of_thread_at<D>(g, batch_plane<D>(g), v)) return;
  cheb_init_at<D, T, TB>(v, sD, a.b, a.bscale, a.r, a.d, a.inv_th);
}
template <int D, typename T, typename TO>
__global__ void __launch_bounds__(BX) k_cheb_last_b(Batch<ChebLastItem<T, TO>> B, Geom g) {
  OK_LEVEL_SMEM(D, T);
  const ChebLastItem<T, TO>& a = B.a[batch_problem<D>(g)];
  stage_level<D, T>(sW, sD, a.r ? a.W : (const T*)nullptr, (const T*)nullptr);
  Vtx<D> v;
  if (!vertex_of_thread_at<D>(g, batch_plane<D>(g), v)) return;
  cheb_last_at<D, T, TO>(g, v, sW, a.x, a.r, a.din, a.first != 0, a.out, a.oscale);
}
template <int D, typename T>
__global__ void __launch_bounds__(BX) k_restrict_b(Batch<TransferItem<T>> B, Geom gf, Geom gc) {
  OK_LEVEL_SMEM(D, T);
  const TransferItem<T>& a = B.a[batch_problem<D>(gc)];
  stage_level<D, T>(sW, sD, (const T*)nullptr, a.dinv);
  Vtx<D> v;
  if (!vertex_of_thread_at<D>(gc, batch_plane<D>(gc), v)) return;
  restrict_at<D, T>(gf, v, a.fine, a.coarse);
  if (a.dinv) cheb_init_at<D, T, T>(v, sD, a.coarse, (T)1, a.r, a.d, a.inv_th);
}
template <int D, typename T>
__global__ void __launch_bounds__(BX) k_prolong_add_b(Batch<TransferItem<T>> B, Geom gf, Geom gc) {
  pdl_entry();
  const TransferItem<T>& a = B.a[batch_problem<D>(gf)];
  Vtx<D> v;
  if (!vertex_of_thread_at<D>(gf, batch_plane<D>(gf), v)) return;
  prolong_add_at<D, T>(gc, v, a.fine, a.coarse, (const T*)a.dc);
}
template <typename T>
__global__ void __launch_bounds__(512) k_coarse_solve_b(Batch<GemvItem<T>> B, long long nc) {
  pdl_entry();
  const GemvItem<T>& a = B.a[blockIdx.x];
  coarse_rows<T>(nc, a.A, a.b, a.x, threadIdx.x >> 5, blockDim.x >> 5);
}

// ---------------------------------------------------------------------------
// fused coarse V-cycle: levels Lc..L in one thread block, vectors in shared
// memory; the same sequence of steps as Prec::vcycle on the host, each step a
// block-stride loop followed by __syncthreads().
// ---------------------------------------------------------------------------
// vertex record of linear index i (< 2^16) without division: i / (n+1) = umulhi(i, mul)
template <int D>
__device__ __forceinline__ void vertex_fast(const Geom& g, unsigned mul, int i, Vtx<D>& v) {
  const int n1 = g.n1;
  const int q = (int)__umulhi((unsigned)i, mul);
  v.idx = i;
  v.p[0] = i - q * n1;
  if (D == 3) {
    const int q2 = (int)__umulhi((unsigned)q, mul);
    v.p[1] = q - q2 * n1;
    v.p[2] = q2;
  } else {
    v.p[1] = q;
    v.p[2] = 0;
  }
  v.c[0] = axis_class(v.p[0], g.n);
  v.c[1] = axis_class(v.p[1], g.n);
  v.c[2] = D == 3 ? axis_class(v.p[2], g.n) : 1;
  v.cls = v.c[0] + 3 * v.c[1] + (D == 3 ? 9 * v.c[2] : 0);
}

#define OK_FOR_VERTICES(L, G, V, BODY)                                               \
  for (int _i = threadIdx.x; _i < (int)(G).nv; _i += blockDim.x) {                   \
    Vtx<D> V;                                                                        \
    vertex_fast<D>((G), a.mul[L], _i, V);                                            \
    BODY;                                                                            \
  }                                                                                  \
  __syncthreads();

// interior vertex number i (0 <= i < (n-1)^D): every class is the interior
// one, known at compile time, so the stencil needs no validity tests
template <int D>
__device__ __forceinline__ void interior_vertex(const Geom& g, unsigned mulI, int i, Vtx<D>& v) {
  const int w = g.n - 1;
  const int q = (w == 1) ? i : (int)__umulhi((unsigned)i, mulI);
  v.p[0] = i - q * w + 1;
  if (D == 3) {
    const int q2 = (w == 1) ? q : (int)__umulhi((unsigned)q, mulI);
    v.p[1] = q - q2 * w + 1;
    v.p[2] = q2 + 1;
  } else {
    v.p[1] = q + 1;
    v.p[2] = 0;
  }
  v.idx = v.p[0] + g.sy * v.p[1] + g.sz * v.p[2];
  v.c[0] = v.c[1] = v.c[2] = 1;
  v.cls = D == 2 ? 4 : 13;
}

// BODY over all vertices: the interior ones first (fast path), then the
// boundary ones; each vertex exactly once, then a barrier
#define OK_FOR_SPLIT(L, G, V, BODY)                                                    \
  {                                                                                    \
    const int _w = (G).n - 1;                                                          \
    const int _ni = D == 3 ? _w * _w * _w : _w * _w;                                   \
    for (int _i = threadIdx.x; _i < _ni; _i += blockDim.x) {                           \
      Vtx<D> V;                                                                        \
      interior_vertex<D>((G), a.mulI[L], _i, V);                                       \
      BODY;                                                                            \
    }                                                                                  \
    for (int _i = threadIdx.x; _i < (int)(G).nv; _i += blockDim.x) {                   \
      Vtx<D> V;                                                                        \
      vertex_fast<D>((G), a.mul[L], _i, V);                                            \
      if (V.cls != (D == 2 ? 4 : 13)) {                                                \
        BODY;                                                                          \
      }                                                                                \
    }                                                                                  \
  }                                                                                    \
  __syncthreads();

template <int D, typename T>
__device__ void fused_smooth(const CoarseArgs<T>& a, int l, T* sm, bool x_zero, int nu, bool want_r) {
  const Geom& g = a.g[l];
  const long long nv = g.nv;
  T* X = sm + a.off[l];
  T* B = X + nv;
  T* R = B + nv;
  T* Dd[2] = {R + nv, R + 2 * nv};
  const T* W = sm + a.toff[l];                        // shared-memory copies of the tables
  const T* dv = W + Topo<D>::NCLASS * Topo<D>::NOFF;
  if (x_zero) {
    OK_FOR_SPLIT(l, g, v, (cheb_init_at<D, T, T>(v, dv, B, (T)1, R, Dd[0], a.inv_th)))
  } else {
    OK_FOR_SPLIT(l, g, v, (resid_init_at<D, T>(g, v, W, dv, B, X, R, Dd[0], a.inv_th)))
  }
  int cur = 0;
  for (int k = 0; k + 1 < nu; ++k) {
    const bool first = x_zero && k == 0;
    OK_FOR_SPLIT(l, g, v, (cheb_step_at<D, T>(g, v, W, dv, X, R, Dd[cur], Dd[1 - cur], a.c1[k], a.c2[k], first)))
    cur ^= 1;
  }
  const bool first = x_zero && nu == 1;
  OK_FOR_SPLIT(l, g, v, (cheb_last_at<D, T, T>(g, v, W, X, want_r ? R : (T*)nullptr, Dd[cur], first, (T*)nullptr,
                                               (T)1)))
}

template <int D, typename T>
__device__ __forceinline__ void coarse_vcycle_body(const CoarseArgs<T>& a, const T* __restrict__ b_in,
                                                   const T* x_in, T* x_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int L = a.nlev - 1;
  {
    T* X0 = sm + a.off[0];
    T* B0 = X0 + a.g[0].nv;
    // loads first (all in flight), then the shared-memory stores; the fused
    // part holds at most 200 KB / (5 * 4 B) = 10240 vertices on level 0
    const int nv0 = (int)a.g[0].nv;
    constexpr int NL = 10;
    T br[NL], xr[NL];
#pragma unroll
    for (int k = 0; k < NL; ++k) {
      const int i = threadIdx.x + k * 1024;
      br[k] = i < nv0 ? b_in[i] : (T)0;
      xr[k] = (x_in && i < nv0) ? x_in[i] : (T)0;
    }
#pragma unroll
    for (int k = 0; k < NL; ++k) {
      const int i = threadIdx.x + k * 1024;
      if (i < nv0) {
        B0[i] = br[k];
        if (x_in) X0[i] = xr[k];
      }
    }
    for (int i = threadIdx.x + NL * 1024; i < nv0; i += blockDim.x) {   // (not reached with the budget above)
      B0[i] = b_in[i];
      if (x_in) X0[i] = x_in[i];
    }
    constexpr int NT = Topo<D>::NCLASS * Topo<D>::NOFF;
    for (int l = 0; l <= L; ++l)
      for (int i = threadIdx.x; i < NT + Topo<D>::NCLASS; i += blockDim.x)
        sm[a.toff[l] + i] = i < NT ? a.W[l][i] : a.dinv[l][i - NT];
    __syncthreads();
  }
  // descend
  for (int l = 0; l < L; ++l) {
    fused_smooth<D, T>(a, l, sm, l > 0 || x_in == nullptr, a.nu_pre, true);
    const Geom& gc = a.g[l + 1];
    T* Rf = sm + a.off[l] + 2 * a.g[l].nv;
    T* Bc = sm + a.off[l + 1] + gc.nv;
    OK_FOR_SPLIT(l + 1, gc, v, (restrict_at<D, T>(a.g[l], v, Rf, Bc)))
  }
  // coarsest: exact
  {
    T* Xc = sm + a.off[L];
    coarse_rows<T>(a.g[L].nv, a.Ainv, Xc + a.g[L].nv, Xc, threadIdx.x >> 5, blockDim.x >> 5);
    __syncthreads();
  }
  // ascend
  for (int l = L - 1; l >= 0; --l) {
    const Geom& g = a.g[l];
    T* Xf = sm + a.off[l];
    const T* Xc = sm + a.off[l + 1];
    OK_FOR_VERTICES(l, g, v, (prolong_add_at<D, T>(a.g[l + 1], v, Xf, Xc)))
    fused_smooth<D, T>(a, l, sm, false, a.nu_post, false);
  }
  for (long long i = threadIdx.x; i < a.g[0].nv; i += blockDim.x) x_out[i] = sm[a.off[0] + i];
}
template <int D, typename T>
__global__ void __launch_bounds__(1024) k_coarse_vcycle(CoarseArgs<T> a, const T* __restrict__ b_in,
                                                        const T* x_in, T* x_out) {
  pdl_entry();   // x_in may equal x_out
  coarse_vcycle_body<D, T>(a, b_in, x_in, x_out);
}
// batched: one block per problem (the problems' level tables differ)
template <int D, typename T>
__global__ void __launch_bounds__(1024) k_coarse_vcycle_b(Batch<CoarseVItem<T>> B) {
  pdl_entry();
  const CoarseVItem<T>& it = B.a[blockIdx.x];
  coarse_vcycle_body<D, T>(*it.a, it.b_in, it.x_in, it.x_out);
}

template <int D, typename T, typename TX, typename TY>
__global__ void __launch_bounds__(BX) k_op_apply(Geom g, const T* __restrict__ W, int axis_only,
                                                 const TX* __restrict__ x, TY* __restrict__ y, T alpha,
                                                 const TY* __restrict__ y0, T beta) {
  using Tp = Topo<D>;
  OK_LEVEL_SMEM(D, T);
  stage_level<D, T>(sW, sD, W, (const T*)nullptr);
  Vtx<D> v;
  if (!vertex_of_thread<D>(g, v)) return;
  T xs[Tp::NOFF];
  load_nb<D>(x, g, v, xs);
  T acc = axis_only ? dot_w<D, Tp::NAX>(sW, v.cls, xs) : dot_w<D, Tp::NOFF>(sW, v.cls, xs);
  acc *= alpha;
  if (y0) acc = fma(beta, (T)y0[v.idx], acc);
  y[v.idx] = (TY)acc;
}

template <int D>
__global__ void k_dense_from_table(Geom g, const double* __restrict__ W, double* __restrict__ A) {
  pdl_entry();
  using Tp = Topo<D>;
  Vtx<D> v;
  if (!vertex_of_thread<D>(g, v)) return;
  static_for<0, Tp::NOFF>([&](auto O) {
    constexpr int o = decltype(O)::value;
    if (nb_valid<D, o>(v.c)) A[v.idx * g.nv + v.idx + nb_delta<D, o>(g)] = W[v.cls * Tp::NOFF + o];
  });
}

// Gauss--Jordan on the n x 2n array [A | I] without pivoting (A is SPD): per
// pivot p one single-block kernel scales row p and saves the column factors,
// then one grid-wide kernel eliminates column p from every other row.
__global__ void k_gj_init(long long n, const double* __restrict__ A, double* __restrict__ w) {
  pdl_entry();
  const long long n2 = 2 * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n * n2;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / n2, c = e % n2;
    w[e] = c < n ? A[r * n + c] : (c - n == r ? 1.0 : 0.0);
  }
}
__global__ void __launch_bounds__(1024) k_gj_pivot(long long n, double* __restrict__ w, double* __restrict__ col,
                                                   long long p) {
  pdl_entry();
  const long long n2 = 2 * n;
  const double piv = w[p * n2 + p];
  __syncthreads();
  for (long long c = threadIdx.x; c < n2; c += blockDim.x) w[p * n2 + c] /= piv;
  for (long long r = threadIdx.x; r < n; r += blockDim.x) col[r] = (r == p) ? 0.0 : w[r * n2 + p];
}
__global__ void k_gj_elim(long long n, double* __restrict__ w, const double* __restrict__ col, long long p) {
  pdl_entry();
  const long long n2 = 2 * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n * n2;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / n2, c = e % n2;
    if (r != p) w[e] -= col[r] * w[p * n2 + c];
  }
}
__global__ void k_gj_extract(long long n, const double* __restrict__ w, double* __restrict__ Ainv) {
  pdl_entry();
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n * n;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / n, c = e % n;
    Ainv[e] = w[r * 2 * n + n + c];
  }
}

// x = Ainv b by many blocks, a warp per row (gemv_row of ok_stencil.cuh on the
// zero-padded inverse; b staged in shared memory).
constexpr int GEMV_WARPS = 8;

template <typename T>
__device__ __forceinline__ void coarse_gemv_body(long long nc, long long ld, const T* __restrict__ A,
                                                 const T* __restrict__ b, T* __restrict__ x) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sb = reinterpret_cast<T*>(smraw);
  const long long r = (long long)blockIdx.x * GEMV_WARPS + (threadIdx.x >> 5);
  typename Vec16<T>::type a0[GEMV_NPL];               // first chunk of the row: A is fixed at setup
  if (r < nc) gemv_load<T>(reinterpret_cast<const typename Vec16<T>::type*>(A + r * ld), ld / Vec16<T>::E, 0, a0);
  pdl_wait();
  gemv_stage_b<T, false>(nc, ld, b, sb);
  __syncthreads();
  if (r >= nc) return;
  const T acc = gemv_finish<T>(ld, A, sb, r, a0);
  if ((threadIdx.x & 31) == 0) x[r] = acc;
}
template <typename T>
__global__ void __launch_bounds__(GEMV_WARPS * 32) k_coarse_gemv(long long nc, long long ld, const T* __restrict__ A,
                                                                const T* __restrict__ b, T* __restrict__ x) {
  pdl_launch_dependents();
  coarse_gemv_body<T>(nc, ld, A, b, x);
}
template <typename T>
__global__ void __launch_bounds__(GEMV_WARPS * 32) k_coarse_gemv_b(Batch<GemvItem<T>> B, long long nc, long long ld) {
  pdl_launch_dependents();
  const GemvItem<T>& a = B.a[blockIdx.y];
  coarse_gemv_body<T>(nc, ld, a.A, a.b, a.x);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
#define OK_DISPATCH(dim, KERNEL, ...)                           \
  do {                                                          \
    if ((dim) == 2) KERNEL<2 __VA_ARGS__;                       \
    else KERNEL<3 __VA_ARGS__;                                  \
  } while (0)

template <typename T, typename TB>
void launch_cheb_init(int dim, const Geom& g, const T* dinv, const TB* b, T bscale, T* r, T* d, T inv_th,
                      cudaStream_t s) {
  if (dim == 2) launch_k(k_cheb_init<2, T, TB>, grid_of(2, g), BX, 0, s, g, dinv, b, bscale, r, d, inv_th);
  else launch_k(k_cheb_init<3, T, TB>, grid_of(3, g), BX, 0, s, g, dinv, b, bscale, r, d, inv_th);
}
template <typename T>
void launch_resid_init(int dim, const Geom& g, const T* W, const T* dinv, const T* b, const T* x, T* r, T* d,
                       T inv_th, cudaStream_t s) {
  if (dim == 2) launch_k(k_resid_init<2, T>, grid_of(2, g), BX, 0, s, g, W, dinv, b, x, r, d, inv_th);
  else launch_k(k_resid_init<3, T>, grid_of(3, g), BX, 0, s, g, W, dinv, b, x, r, d, inv_th);
}
template <typename T>
void launch_cheb_step(int dim, const Geom& g, const T* W, const T* dinv, T* x, T* r, const T* d_in, T* d_out,
                      T c1, T c2, bool first, cudaStream_t s) {
  if (dim == 2) launch_k(k_cheb_step<2, T>, grid_of(2, g), BX, 0, s, g, W, dinv, x, r, d_in, d_out, c1, c2, first);
  else launch_k(k_cheb_step<3, T>, grid_of(3, g), BX, 0, s, g, W, dinv, x, r, d_in, d_out, c1, c2, first);
}
template <typename T, typename TO>
void launch_cheb_last(int dim, const Geom& g, const T* W, T* x, T* r, const T* d_in, bool first, TO* out,
                      T oscale, cudaStream_t s) {
  if (dim == 2) launch_k(k_cheb_last<2, T, TO>, grid_of(2, g), BX, 0, s, g, W, x, r, d_in, first, out, oscale);
  else launch_k(k_cheb_last<3, T, TO>, grid_of(3, g), BX, 0, s, g, W, x, r, d_in, first, out, oscale);
}
template <typename T>
void launch_restrict(int dim, const Geom& gf, const Geom& gc, const T* rf, T* bc, cudaStream_t s,
                     const T* dinv, T* r, T* d, T inv_th) {
  if (dim == 2) launch_k(k_restrict<2, T>, grid_of(2, gc), BX, 0, s, gf, gc, rf, bc, dinv, r, d, inv_th);
  else launch_k(k_restrict<3, T>, grid_of(3, gc), BX, 0, s, gf, gc, rf, bc, dinv, r, d, inv_th);
}
template <typename T>
void launch_prolong_add(int dim, const Geom& gf, const Geom& gc, T* xf, const T* xc, cudaStream_t s, const T* dc) {
  if (dim == 2) launch_k(k_prolong_add<2, T>, grid_of(2, gf), BX, 0, s, gf, gc, xf, xc, dc);
  else launch_k(k_prolong_add<3, T>, grid_of(3, gf), BX, 0, s, gf, gc, xf, xc, dc);
}
template <typename T>
void launch_coarse_solve(long long nc, const T* Ainv, const T* b, T* x, cudaStream_t s) {
  launch_k(k_coarse_solve<T>, 1, 512, 0, s, nc, Ainv, b, x);
}
long long gemv_ld(long long nc, size_t elem) {
  const long long e = 16 / (long long)elem;
  return (nc + e - 1) / e * e;
}
template <typename T>
void launch_coarse_gemv(long long nc, long long ld, const T* Ainv, const T* b, T* x, cudaStream_t s) {
  const unsigned blocks = (unsigned)((nc + GEMV_WARPS - 1) / GEMV_WARPS);
  launch_k(k_coarse_gemv<T>, blocks, GEMV_WARPS * 32, gemv_staged<T>(ld) * sizeof(T), s, nc, ld, Ainv, b, x);
}
template <typename T>
cudaError_t prepare_coarse_gemv(long long nc) {
  // per-kernel limit shared by all handles: the largest coarsest level's need
  (void)nc;
  const size_t need = (size_t)gemv_staged<T>(gemv_ld(COARSE_NC_MAX, sizeof(T))) * sizeof(T);
  cudaError_t e = cudaFuncSetAttribute(k_coarse_gemv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)std::max(need, (size_t)48 * 1024));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_coarse_gemv_b<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)std::max(need, (size_t)48 * 1024));
}
template <typename T, typename TX, typename TY>
void launch_op_apply(int dim, const Geom& g, const T* W, bool axis_only, const TX* x, TY* y, T alpha,
                     const TY* y0, T beta, cudaStream_t s) {
  if (dim == 2) launch_k(k_op_apply<2, T, TX, TY>, grid_of(2, g), BX, 0, s, g, W, axis_only, x, y, alpha, y0, beta);
  else launch_k(k_op_apply<3, T, TX, TY>, grid_of(3, g), BX, 0, s, g, W, axis_only, x, y, alpha, y0, beta);
}
template <typename T>
void launch_coarse_vcycle(int dim, const CoarseArgs<T>& a, size_t smem, const T* b_in, const T* x_in, T* x_out,
                          cudaStream_t s) {
  if (dim == 2) launch_k(k_coarse_vcycle<2, T>, 1, 1024, smem, s, a, b_in, x_in, x_out);
  else launch_k(k_coarse_vcycle<3, T>, 1, 1024, smem, s, a, b_in, x_in, x_out);
}
template <typename T>
cudaError_t prepare_coarse_vcycle(int dim, size_t smem) {
  if (smem > COARSE_SMEM_MAX) return cudaErrorInvalidValue;
  const int lim = (int)COARSE_SMEM_MAX;             // shared by all handles: never lowered
  const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
  if (dim == 2) {
    cudaError_t e = cudaFuncSetAttribute(k_coarse_vcycle<2, T>, at, lim);
    return e != cudaSuccess ? e : cudaFuncSetAttribute(k_coarse_vcycle_b<2, T>, at, lim);
  }
  cudaError_t e = cudaFuncSetAttribute(k_coarse_vcycle<3, T>, at, lim);
  return e != cudaSuccess ? e : cudaFuncSetAttribute(k_coarse_vcycle_b<3, T>, at, lim);
}
template void launch_coarse_vcycle<double>(int, const CoarseArgs<double>&, size_t, const double*, const double*,
                                           double*, cudaStream_t);
template void launch_coarse_vcycle<float>(int, const CoarseArgs<float>&, size_t, const float*, const float*, float*,
                                          cudaStream_t);
template cudaError_t prepare_coarse_vcycle<double>(int, size_t);
template cudaError_t prepare_coarse_vcycle<float>(int, size_t);

void launch_dense_from_table(int dim, const Geom& g, const double* W, double* A, cudaStream_t s) {
  if (dim == 2) launch_k(k_dense_from_table<2>, grid_of(2, g), BX, 0, s, g, W, A);
  else launch_k(k_dense_from_table<3>, grid_of(3, g), BX, 0, s, g, W, A);
}
// work: n x 2n array followed by n column factors
void launch_gauss_jordan(long long n, const double* A, double* work, double* Ainv, cudaStream_t s) {
  double* col = work + 2 * n * n;
  const unsigned blocks = (unsigned)std::min<long long>((2 * n * n + 255) / 256, 4096);
  launch_k(k_gj_init, blocks, 256, 0, s, n, A, work);
  for (long long p = 0; p < n; ++p) {
    launch_k(k_gj_pivot, 1, 1024, 0, s, n, work, col, p);
    launch_k(k_gj_elim, blocks, 256, 0, s, n, work, col, p);
  }
  launch_k(k_gj_extract, blocks, 256, 0, s, n, work, Ainv);
}

// ---- batched launchers ----------------------------------------------------
template <int D>
static inline dim3 grid_b(const Geom& g, int count) {
  return dim3((unsigned)(((long long)g.n1 * g.n1 + BX - 1) / BX), 1, (D == 3 ? g.n1 : 1) * count);
}
template <typename I>
static inline Batch<I> pack(const I* items, int count) {
  Batch<I> B;
  for (int i = 0; i < count; ++i) B.a[i] = items[i];
  return B;
}
template <typename T, typename TB>
void launch_cheb_init_b(int dim, const Geom& g, const ChebInitItem<T, TB>* items, int count, cudaStream_t s) {
  auto B = pack(items, count);
  if (dim == 2) launch_k(k_cheb_init_b<2, T, TB>, grid_b<2>(g, count), BX, 0, s, B, g);
  else launch_k(k_cheb_init_b<3, T, TB>, grid_b<3>(g, count), BX, 0, s, B, g);
}
template <typename T, typename TO>
void launch_cheb_last_b(int dim, const Geom& g, const ChebLastItem<T, TO>* items, int count, cudaStream_t s) {
  auto B = pack(items, count);
  if (dim == 2) launch_k(k_cheb_last_b<2, T, TO>, grid_b<2>(g, count), BX, 0, s, B, g);
  else launch_k(k_cheb_last_b<3, T, TO>, grid_b<3>(g, count), BX, 0, s, B, g);
}
template <typename T>
void launch_restrict_b(int dim, const Geom& gf, const Geom& gc, const TransferItem<T>* items, int count,
                       cudaStream_t s) {
  auto B = pack(items, count);
  if (dim == 2) launch_k(k_restrict_b<2, T>, grid_b<2>(gc, count), BX, 0, s, B, gf, gc);
  else launch_k(k_restrict_b<3, T>, grid_b<3>(gc, count), BX, 0, s, B, gf, gc);
}
template <typename T>
void launch_prolong_add_b(int dim, const Geom& gf, const Geom& gc, const TransferItem<T>* items, int count,
                          cudaStream_t s) {
  auto B = pack(items, count);
  if (dim == 2) launch_k(k_prolong_add_b<2, T>, grid_b<2>(gf, count), BX, 0, s, B, gf, gc);
  else launch_k(k_prolong_add_b<3, T>, grid_b<3>(gf, count), BX, 0, s, B, gf, gc);
}
template <typename T>
void launch_coarse_solve_b(long long nc, long long ld, bool gemv, const GemvItem<T>* items, int count,
                           cudaStream_t s) {
  auto B = pack(items, count);
  if (gemv) {
    const unsigned blocks = (unsigned)((nc + GEMV_WARPS - 1) / GEMV_WARPS);
    launch_k(k_coarse_gemv_b<T>, dim3(blocks, count), GEMV_WARPS * 32, gemv_staged<T>(ld) * sizeof(T), s, B, nc, ld);
  } else {
    launch_k(k_coarse_solve_b<T>, count, 512, 0, s, B, nc);
  }
}
template <typename T>
void launch_coarse_vcycle_b(int dim, const CoarseVItem<T>* items, int count, size_t smem, cudaStream_t s) {
  auto B = pack(items, count);
  if (dim == 2) launch_k(k_coarse_vcycle_b<2, T>, count, 1024, smem, s, B);
  else launch_k(k_coarse_vcycle_b<3, T>, count, 1024, smem, s, B);
}
#define OK_INST_B(T)                                                                                          \
  template void launch_restrict_b<T>(int, const Geom&, const Geom&, const TransferItem<T>*, int, cudaStream_t); \
  template void launch_prolong_add_b<T>(int, const Geom&, const Geom&, const TransferItem<T>*, int,          \
                                        cudaStream_t);                                                        \
  template void launch_coarse_solve_b<T>(long long, long long, bool, const GemvItem<T>*, int, cudaStream_t);  \
  template void launch_coarse_vcycle_b<T>(int, const CoarseVItem<T>*, int, size_t, cudaStream_t);             \
  template void launch_cheb_init_b<T, T>(int, const Geom&, const ChebInitItem<T, T>*, int, cudaStream_t);     \
  template void launch_cheb_last_b<T, T>(int, const Geom&, const ChebLastItem<T, T>*, int, cudaStream_t);
OK_INST_B(float)
OK_INST_B(double)
template void launch_cheb_init_b<float, double>(int, const Geom&, const ChebInitItem<float, double>*, int,
                                                cudaStream_t);
template void launch_cheb_last_b<float, __half>(int, const Geom&, const ChebLastItem<float, __half>*, int,
                                                cudaStream_t);

#define OK_INST_T(T)                                                                                          \
  template void launch_resid_init<T>(int, const Geom&, const T*, const T*, const T*, const T*, T*, T*, T,      \
                                     cudaStream_t);                                                            \
  template void launch_cheb_step<T>(int, const Geom&, const T*, const T*, T*, T*, const T*, T*, T, T, bool,    \
                                    cudaStream_t);                                                             \
  template void launch_restrict<T>(int, const Geom&, const Geom&, const T*, T*, cudaStream_t, const T*, T*, T*, \
                                   T);                                                                        \
  template void launch_prolong_add<T>(int, const Geom&, const Geom&, T*, const T*, cudaStream_t, const T*);    \
  template void launch_coarse_solve<T>(long long, const T*, const T*, T*, cudaStream_t);                  \
  template void launch_coarse_gemv<T>(long long, long long, const T*, const T*, T*, cudaStream_t);        \
  template cudaError_t prepare_coarse_gemv<T>(long long);

OK_INST_T(double)
OK_INST_T(float)

template void launch_cheb_init<double, double>(int, const Geom&, const double*, const double*, double, double*,
                                               double*, double, cudaStream_t);
template void launch_cheb_init<float, double>(int, const Geom&, const float*, const double*, float, float*, float*,
                                              float, cudaStream_t);
template void launch_cheb_init<float, float>(int, const Geom&, const float*, const float*, float, float*, float*,
                                             float, cudaStream_t);
template void launch_cheb_last<double, double>(int, const Geom&, const double*, double*, double*, const double*,
                                               bool, double*, double, cudaStream_t);
template void launch_cheb_last<float, float>(int, const Geom&, const float*, float*, float*, const float*, bool,
                                             float*, float, cudaStream_t);
template void launch_cheb_last<float, __half>(int, const Geom&, const float*, float*, float*, const float*, bool,
                                              __half*, float, cudaStream_t);
template void launch_cheb_last<double, float>(int, const Geom&, const double*, double*, double*, const double*,
                                              bool, float*, double, cudaStream_t);
template void launch_cheb_last<float, double>(int, const Geom&, const float*, float*, float*, const float*, bool,
                                              double*, float, cudaStream_t);
template void launch_op_apply<double, double, double>(int, const Geom&, const double*, bool, const double*,
                                                      double*, double, const double*, double, cudaStream_t);
template void launch_op_apply<float, float, float>(int, const Geom&, const float*, bool, const float*, float*,
                                                   float, const float*, float, cudaStream_t);
template void launch_op_apply<double, float, double>(int, const Geom&, const double*, bool, const float*,
                                                     double*, double, const double*, double, cudaStream_t);

}  // namespace okg
