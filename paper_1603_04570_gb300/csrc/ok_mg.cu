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
#include "ok_internal.cuh"
#include "ok_kernels.h"

namespace okg {

static constexpr int BX = 128;

static inline dim3 grid_of(int dim, const Geom& g) {
  return dim3((g.n1 + BX - 1) / BX, g.n1, dim == 3 ? g.n1 : 1);
}

template <int D, typename T, typename TB>
__global__ void __launch_bounds__(BX) k_cheb_init(Geom g, const T* __restrict__ dinv, const TB* __restrict__ b,
                                                  T bscale, T* __restrict__ r, T* __restrict__ d, T inv_th) {
  Vtx<D> v;
  if (!vertex_of_thread<D>(g, v)) return;
  T rr = (T)b[v.idx] * bscale;
  r[v.idx] = rr;
  d[v.idx] = dinv[v.cls] * rr * inv_th;
}

template <int D, typename T>
__global__ void __launch_bounds__(BX) k_resid_init(Geom g, const T* __restrict__ W, const T* __restrict__ dinv,
                                                   const T* __restrict__ b, const T* __restrict__ x,
                                                   T* __restrict__ r, T* __restrict__ d, T inv_th) {
  using Tp = Topo<D>;
  Vtx<D> v;
  if (!vertex_of_thread<D>(g, v)) return;
  T xs[Tp::NOFF];
  load_nb<D>(x, g, v, xs);
  T rr = b[v.idx] - dot_w<D, Tp::NOFF>(W, v.cls, xs);
  r[v.idx] = rr;
  d[v.idx] = dinv[v.cls] * rr * inv_th;
}

template <int D, typename T>
__global__ void __launch_bounds__(BX) k_cheb_step(Geom g, const T* __restrict__ W, const T* __restrict__ dinv,
                                                  T* __restrict__ x, T* __restrict__ r, const T* __restrict__ din,
                                                  T* __restrict__ dout, T c1, T c2, int first) {
  using Tp = Topo<D>;
  Vtx<D> v;
  if (!vertex_of_thread<D>(g, v)) return;
  T ds[Tp::NOFF];
  load_nb<D>(din, g, v, ds);
  x[v.idx] = (first ? (T)0 : x[v.idx]) + ds[0];
  T rr = r[v.idx] - dot_w<D, Tp::NOFF>(W, v.cls, ds);
  r[v.idx] = rr;
  dout[v.idx] = c1 * ds[0] + c2 * (dinv[v.cls] * rr);
}

template <int D, typename T, typename TO>
__global__ void __launch_bounds__(BX) k_cheb_last(Geom g, const T* __restrict__ W, T* __restrict__ x,
                                                  T* __restrict__ r, const T* __restrict__ din, int first,
                                                  TO* __restrict__ out, T oscale) {
  using Tp = Topo<D>;
  Vtx<D> v;
  if (!vertex_of_thread<D>(g, v)) return;
  T xx;
  if (r) {
    T ds[Tp::NOFF];
    load_nb<D>(din, g, v, ds);
    xx = (first ? (T)0 : x[v.idx]) + ds[0];
    r[v.idx] = r[v.idx] - dot_w<D, Tp::NOFF>(W, v.cls, ds);
  } else {
    xx = (first ? (T)0 : x[v.idx]) + din[v.idx];
  }
  x[v.idx] = xx;
  if (out) out[v.idx] = (TO)(xx * oscale);
}

template <int D, typename T>
__global__ void __launch_bounds__(BX) k_restrict(Geom gf, Geom gc, const T* __restrict__ rf, T* __restrict__ bc) {
  using Tp = Topo<D>;
  Vtx<D> v;                               // coarse vertex
  if (!vertex_of_thread<D>(gc, v)) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = D == 3 ? blockIdx.z : 0;
  long long fc = 2LL * i + gf.sy * (2LL * j) + gf.sz * (2LL * k);
  T acc = (T)0;
  static_for<1, Tp::NOFF>([&](auto O) {
    constexpr int o = decltype(O)::value;
    if (nb_valid<D, o>(v.c)) acc += rf[fc + nb_delta<D, o>(gf)];
  });
  bc[v.idx] = rf[fc] + (T)0.5 * acc;
}

template <int D, typename T>
__global__ void __launch_bounds__(BX) k_prolong_add(Geom gf, Geom gc, T* __restrict__ xf, const T* __restrict__ xc) {
  Vtx<D> v;                               // fine vertex
  if (!vertex_of_thread<D>(gf, v)) return;
  int f[3] = {(int)(blockIdx.x * blockDim.x + threadIdx.x), (int)blockIdx.y, D == 3 ? (int)blockIdx.z : 0};
  long long ci = 0, cj = 0;
  bool mid = false;
  long long st[3] = {1, gc.sy, gc.sz};
#pragma unroll
  for (int a = 0; a < D; ++a) {
    ci += (long long)(f[a] >> 1) * st[a];
    cj += (long long)((f[a] >> 1) + (f[a] & 1)) * st[a];
    mid = mid || (f[a] & 1);
  }
  T add = mid ? (T)0.5 * (xc[ci] + xc[cj]) : xc[ci];
  xf[v.idx] += add;
}

// one block; warp per row
template <typename T>
__global__ void __launch_bounds__(512) k_coarse_solve(long long nc, const T* __restrict__ A, const T* __restrict__ b,
                                                      T* __restrict__ x) {
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (long long r = warp; r < nc; r += nw) {
    T acc = (T)0;
    for (long long c = lane; c < nc; c += 32) acc = fma(A[r * nc + c], b[c], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) x[r] = acc;
  }
}

template <int D, typename T, typename TX, typename TY>
__global__ void __launch_bounds__(BX) k_op_apply(Geom g, const T* __restrict__ W, int axis_only,
                                                 const TX* __restrict__ x, TY* __restrict__ y, T alpha,
                                                 const TY* __restrict__ y0, T beta) {
  using Tp = Topo<D>;
  Vtx<D> v;
  if (!vertex_of_thread<D>(g, v)) return;
  T xs[Tp::NOFF];
  load_nb<D>(x, g, v, xs);
  T acc = axis_only ? dot_w<D, Tp::NAX>(W, v.cls, xs) : dot_w<D, Tp::NOFF>(W, v.cls, xs);
  acc *= alpha;
  if (y0) acc = fma(beta, (T)y0[v.idx], acc);
  y[v.idx] = (TY)acc;
}

template <int D>
__global__ void k_dense_from_table(Geom g, const double* __restrict__ W, double* __restrict__ A) {
  using Tp = Topo<D>;
  Vtx<D> v;
  if (!vertex_of_thread<D>(g, v)) return;
  static_for<0, Tp::NOFF>([&](auto O) {
    constexpr int o = decltype(O)::value;
    if (nb_valid<D, o>(v.c)) A[v.idx * g.nv + v.idx + nb_delta<D, o>(g)] = W[v.cls * Tp::NOFF + o];
  });
}

// Gauss--Jordan on [A | I] without pivoting (A is SPD), one block.
__global__ void __launch_bounds__(1024) k_gauss_jordan(long long n, const double* __restrict__ A,
                                                       double* __restrict__ w, double* __restrict__ Ainv) {
  const long long n2 = 2 * n;
  for (long long e = threadIdx.x; e < n * n2; e += blockDim.x) {
    long long r = e / n2, c = e % n2;
    w[e] = c < n ? A[r * n + c] : (c - n == r ? 1.0 : 0.0);
  }
  extern __shared__ double col[];   // n factors
  __syncthreads();
  for (long long p = 0; p < n; ++p) {
    const double piv = w[p * n2 + p];
    __syncthreads();
    for (long long c = threadIdx.x; c < n2; c += blockDim.x) w[p * n2 + c] /= piv;
    __syncthreads();
    for (long long r = threadIdx.x; r < n; r += blockDim.x) col[r] = (r == p) ? 0.0 : w[r * n2 + p];
    __syncthreads();
    for (long long e = threadIdx.x; e < n * n2; e += blockDim.x) {
      long long r = e / n2, c = e % n2;
      if (r != p) w[e] -= col[r] * w[p * n2 + c];
    }
    __syncthreads();
  }
  for (long long e = threadIdx.x; e < n * n; e += blockDim.x) {
    long long r = e / n, c = e % n;
    Ainv[e] = w[r * n2 + n + c];
  }
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
  if (dim == 2) k_cheb_init<2, T, TB><<<grid_of(2, g), BX, 0, s>>>(g, dinv, b, bscale, r, d, inv_th);
  else k_cheb_init<3, T, TB><<<grid_of(3, g), BX, 0, s>>>(g, dinv, b, bscale, r, d, inv_th);
}
template <typename T>
void launch_resid_init(int dim, const Geom& g, const T* W, const T* dinv, const T* b, const T* x, T* r, T* d,
                       T inv_th, cudaStream_t s) {
  if (dim == 2) k_resid_init<2, T><<<grid_of(2, g), BX, 0, s>>>(g, W, dinv, b, x, r, d, inv_th);
  else k_resid_init<3, T><<<grid_of(3, g), BX, 0, s>>>(g, W, dinv, b, x, r, d, inv_th);
}
template <typename T>
void launch_cheb_step(int dim, const Geom& g, const T* W, const T* dinv, T* x, T* r, const T* d_in, T* d_out,
                      T c1, T c2, bool first, cudaStream_t s) {
  if (dim == 2) k_cheb_step<2, T><<<grid_of(2, g), BX, 0, s>>>(g, W, dinv, x, r, d_in, d_out, c1, c2, first);
  else k_cheb_step<3, T><<<grid_of(3, g), BX, 0, s>>>(g, W, dinv, x, r, d_in, d_out, c1, c2, first);
}
template <typename T, typename TO>
void launch_cheb_last(int dim, const Geom& g, const T* W, T* x, T* r, const T* d_in, bool first, TO* out,
                      T oscale, cudaStream_t s) {
  if (dim == 2) k_cheb_last<2, T, TO><<<grid_of(2, g), BX, 0, s>>>(g, W, x, r, d_in, first, out, oscale);
  else k_cheb_last<3, T, TO><<<grid_of(3, g), BX, 0, s>>>(g, W, x, r, d_in, first, out, oscale);
}
template <typename T>
void launch_restrict(int dim, const Geom& gf, const Geom& gc, const T* rf, T* bc, cudaStream_t s) {
  if (dim == 2) k_restrict<2, T><<<grid_of(2, gc), BX, 0, s>>>(gf, gc, rf, bc);
  else k_restrict<3, T><<<grid_of(3, gc), BX, 0, s>>>(gf, gc, rf, bc);
}
template <typename T>
void launch_prolong_add(int dim, const Geom& gf, const Geom& gc, T* xf, const T* xc, cudaStream_t s) {
  if (dim == 2) k_prolong_add<2, T><<<grid_of(2, gf), BX, 0, s>>>(gf, gc, xf, xc);
  else k_prolong_add<3, T><<<grid_of(3, gf), BX, 0, s>>>(gf, gc, xf, xc);
}
template <typename T>
void launch_coarse_solve(long long nc, const T* Ainv, const T* b, T* x, cudaStream_t s) {
  k_coarse_solve<T><<<1, 512, 0, s>>>(nc, Ainv, b, x);
}
template <typename T, typename TX, typename TY>
void launch_op_apply(int dim, const Geom& g, const T* W, bool axis_only, const TX* x, TY* y, T alpha,
                     const TY* y0, T beta, cudaStream_t s) {
  if (dim == 2) k_op_apply<2, T, TX, TY><<<grid_of(2, g), BX, 0, s>>>(g, W, axis_only, x, y, alpha, y0, beta);
  else k_op_apply<3, T, TX, TY><<<grid_of(3, g), BX, 0, s>>>(g, W, axis_only, x, y, alpha, y0, beta);
}
void launch_dense_from_table(int dim, const Geom& g, const double* W, double* A, cudaStream_t s) {
  if (dim == 2) k_dense_from_table<2><<<grid_of(2, g), BX, 0, s>>>(g, W, A);
  else k_dense_from_table<3><<<grid_of(3, g), BX, 0, s>>>(g, W, A);
}
void launch_gauss_jordan(long long n, const double* A, double* work, double* Ainv, cudaStream_t s) {
  k_gauss_jordan<<<1, 1024, n * sizeof(double), s>>>(n, A, work, Ainv);
}

#define OK_INST_T(T)                                                                                          \
  template void launch_resid_init<T>(int, const Geom&, const T*, const T*, const T*, const T*, T*, T*, T,      \
                                     cudaStream_t);                                                            \
  template void launch_cheb_step<T>(int, const Geom&, const T*, const T*, T*, T*, const T*, T*, T, T, bool,    \
                                    cudaStream_t);                                                             \
  template void launch_restrict<T>(int, const Geom&, const Geom&, const T*, T*, cudaStream_t);                 \
  template void launch_prolong_add<T>(int, const Geom&, const Geom&, T*, const T*, cudaStream_t);              \
  template void launch_coarse_solve<T>(long long, const T*, const T*, T*, cudaStream_t);

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
