// ok_tile.cu -- shared-memory tile kernels with temporal blocking (2D grids).
//
// One thread block owns a TILE x TILE square of vertices of one multigrid
// level and loads it with a halo wide enough to take several dependent steps
// without a grid-wide synchronisation: the halo points are recomputed by the
// neighbouring blocks (redundant work) instead of exchanged.  Every point
// update goes through the per-vertex bodies of ok_stencil.cuh, so the result
// is bitwise the same as the one-kernel-per-step path.
//
//   k_tile_pre   two Chebyshev--Jacobi pre-smoothing steps on S_hat from x
//                (or from zero), the residual, and its restriction P^T r to
//                the coarser level (halo 4);
//   k_tile_post  prolongation x += P x_c and two post-smoothing steps
//                (halo 3), optionally M x (the middle factor of
//                S~^{-1} = S_hat^{-1} M S_hat^{-1}) and a cast of x to an
//                output vector;
//   k_tile_amass q Chebyshev steps on M (A~^{-1} r1, Sec. 3) and the
//                preconditioner's C-step t = r2 - C A~^{-1} r1 (eqn prec)
//                (halo q).
// x is read from one buffer and written to another (ping-pong), because
// other blocks read the old x in their halos while this block writes.
#include "ok_internal.cuh"
#include "ok_kernels.h"
#include "ok_stencil.cuh"

namespace okg {

constexpr int TILE = 32;
constexpr int TILE_THREADS = 256;
constexpr int QTILE = 10;   // mass Chebyshev steps handled by the tile kernel

// A tile of side S = TILE + 2H around the block's owned TILE x TILE vertices.
template <int TL, int S> struct Frame {
  static constexpr int H = (S - TL) / 2;
  int f0x, f0y;    // global coordinates of the first owned vertex
  int n;           // cells per side of the level
  long long gsy;   // global row stride
  Geom lg;         // local geometry (row stride S) for the stencil bodies
};

template <int TL, int S>
__device__ __forceinline__ Frame<TL, S> make_frame(const Geom& g) {
  Frame<TL, S> F;
  F.f0x = blockIdx.x * TL;
  F.f0y = blockIdx.y * TL;
  F.n = g.n;
  F.gsy = g.sy;
  F.lg.n = g.n;
  F.lg.n1 = S;
  F.lg.nv = (long long)S * S;
  F.lg.sy = S;
  F.lg.sz = 0;
  return F;
}

// Is every vertex of the tile (halo included) an interior vertex?
template <int TL, int S>
__device__ __forceinline__ bool tile_interior(const Frame<TL, S>& F) {
  constexpr int H = Frame<TL, S>::H;
  return F.f0x - H >= 1 && F.f0y - H >= 1 && F.f0x - H + S - 1 <= F.n - 1 && F.f0y - H + S - 1 <= F.n - 1;
}

// local (lx, ly) -> vertex record (local index, global coordinates, class);
// INT: the tile is interior, so the class is the interior one everywhere
template <int TL, int S, bool INT>
__device__ __forceinline__ bool tile_vertex(const Frame<TL, S>& F, int lx, int ly, Vtx<2>& v) {
  constexpr int H = Frame<TL, S>::H;
  const int gx = F.f0x - H + lx, gy = F.f0y - H + ly;
  if (!INT && (gx < 0 || gy < 0 || gx > F.n || gy > F.n)) return false;
  v.idx = (long long)ly * S + lx;
  v.p[0] = gx;
  v.p[1] = gy;
  v.p[2] = 0;
  v.c[0] = INT ? 1 : axis_class(gx, F.n);
  v.c[1] = INT ? 1 : axis_class(gy, F.n);
  v.c[2] = 1;
  v.cls = INT ? 4 : v.c[0] + 3 * v.c[1];
  return true;
}
template <int TL, int S>
__device__ __forceinline__ long long gidx(const Frame<TL, S>& F, const Vtx<2>& v) {
  return v.p[0] + F.gsy * v.p[1];
}

// fn(v) for every in-domain vertex of the local square [LO, HI)^2, then a barrier
template <int TL, int S, int LO, int HI, bool INT, typename Fn>
__device__ __forceinline__ void tile_loop(const Frame<TL, S>& F, Fn&& fn) {
  constexpr int W = HI - LO;
  for (int t = threadIdx.x; t < W * W; t += TILE_THREADS) {
    Vtx<2> v;
    if (tile_vertex<TL, S, INT>(F, LO + t % W, LO + t / W, v)) fn(v);
  }
  __syncthreads();
}

// copy a level's class tables into shared memory (read with warp-uniform addresses)
template <typename T>
__device__ __forceinline__ void load_tables(T* sW, T* sD, const T* W, const T* dinv) {
  for (int i = threadIdx.x; i < Topo<2>::NCLASS * Topo<2>::NOFF; i += TILE_THREADS) sW[i] = W[i];
  for (int i = threadIdx.x; i < Topo<2>::NCLASS; i += TILE_THREADS) sD[i] = dinv[i];
}

// ---------------------------------------------------------------------------
// pre-smoothing (2 steps) + restriction
// ---------------------------------------------------------------------------
template <typename T, int TL, bool INT>
__device__ __forceinline__ void tile_pre_body(const TileSmooth<T>& a, const Frame<TL, TL + 8>& F, T* X, T* B, T* R, T* D0,
                                              T* D1, const T* sW, const T* sD, const T* x_in, const T* b,
                                              T* x_out, T* bc) {
  constexpr int S = TL + 8;
  const bool xz = (x_in == nullptr);
  // all global loads of this thread first (in flight together), then the stores
  constexpr int NL = (S * S + TILE_THREADS - 1) / TILE_THREADS;
  T xr[NL], br[NL];
#pragma unroll
  for (int k = 0; k < NL; ++k) {
    const int t = threadIdx.x + k * TILE_THREADS;
    Vtx<2> v;
    xr[k] = (T)0;
    br[k] = (T)0;
    if (t < S * S && tile_vertex<TL, S, INT>(F, t % S, t / S, v)) {
      const long long gi = gidx(F, v);
      br[k] = b[gi];
      if (!xz) xr[k] = x_in[gi];
    }
  }
#pragma unroll
  for (int k = 0; k < NL; ++k) {
    const int t = threadIdx.x + k * TILE_THREADS;
    if (t < S * S) {
      X[t] = xr[k];
      B[t] = br[k];
    }
  }
  __syncthreads();
  const Geom& lg = F.lg;
  const RegW<2, T> rw = reg_weights<2, T>(sW, sD, 4);   // interior class, used when INT
  if (xz)
    tile_loop<TL, S, 1, S - 1, INT>(F, [&](const Vtx<2>& v) {
      if constexpr (INT) cheb_init_r<2, T>(v, rw, B, R, D0, a.inv_th);
      else cheb_init_at<2, T, T>(v, sD, B, (T)1, R, D0, a.inv_th);
    });
  else
    tile_loop<TL, S, 1, S - 1, INT>(F, [&](const Vtx<2>& v) {
      if constexpr (INT) resid_init_r<2, T>(lg, v, rw, B, X, R, D0, a.inv_th);
      else resid_init_at<2, T>(lg, v, sW, sD, B, X, R, D0, a.inv_th);
    });
  tile_loop<TL, S, 2, S - 2, INT>(F, [&](const Vtx<2>& v) {
    if constexpr (INT) cheb_step_r<2, T>(lg, v, rw, X, R, D0, D1, a.c1, a.c2, xz);
    else cheb_step_at<2, T>(lg, v, sW, sD, X, R, D0, D1, a.c1, a.c2, xz);
  });
  tile_loop<TL, S, 3, S - 3, INT>(F, [&](const Vtx<2>& v) {
    if constexpr (INT) cheb_last_r<2, T>(lg, v, rw, X, R, D1, false);
    else cheb_last_at<2, T, T>(lg, v, sW, X, R, D1, false, (T*)nullptr, (T)1);
  });
  // restriction for the coarse vertices whose fine centre this block owns
  const int nc = a.gc.n;
  for (int t = threadIdx.x; t < (TL / 2) * (TL / 2); t += TILE_THREADS) {
    const int cx = blockIdx.x * (TL / 2) + t % (TL / 2), cy = blockIdx.y * (TL / 2) + t / (TL / 2);
    if (!INT && (cx > nc || cy > nc)) continue;
    Vtx<2> vc;
    vc.c[0] = INT ? 1 : axis_class(cx, nc);
    vc.c[1] = INT ? 1 : axis_class(cy, nc);
    vc.c[2] = 1;
    const long long fc = (long long)(2 * cy - F.f0y + Frame<TL, S>::H) * S + (2 * cx - F.f0x + Frame<TL, S>::H);
    T acc = (T)0;
    static_for<1, Topo<2>::NOFF>([&](auto O) {
      constexpr int o = decltype(O)::value;
      if (nb_valid<2, o>(vc.c)) acc += R[fc + nb_delta<2, o>(lg)];
    });
    bc[cx + a.gc.sy * cy] = fma((T)0.5, acc, R[fc]);
  }
  tile_loop<TL, S, Frame<TL, S>::H, Frame<TL, S>::H + TL, INT>(F, [&](const Vtx<2>& v) { x_out[gidx(F, v)] = X[v.idx]; });
}

template <typename T, int TL>
__global__ void __launch_bounds__(TILE_THREADS) k_tile_pre(TileSmooth<T> a, const T* __restrict__ x_in,
                                                           const T* __restrict__ b, T* __restrict__ x_out,
                                                           T* __restrict__ bc) {
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int S = TL + 8, SS = S * S;
  const Frame<TL, S> F = make_frame<TL, S>(a.g);
  T* X = reinterpret_cast<T*>(smraw);
  T* B = X + SS;
  T* R = B + SS;
  T* D0 = R + SS;
  T* D1 = D0 + SS;
  T* sW = D1 + SS;
  T* sD = sW + Topo<2>::NCLASS * Topo<2>::NOFF;
  load_tables<T>(sW, sD, a.W, a.dinv);
  if (tile_interior(F)) tile_pre_body<T, TL, true>(a, F, X, B, R, D0, D1, sW, sD, x_in, b, x_out, bc);
  else tile_pre_body<T, TL, false>(a, F, X, B, R, D0, D1, sW, sD, x_in, b, x_out, bc);
}

// ---------------------------------------------------------------------------
// prolongation + post-smoothing (2 steps) [+ M x] [+ cast of x]
// ---------------------------------------------------------------------------
template <typename T, typename TO, int TL, bool INT>
__device__ __forceinline__ void tile_post_body(const TileSmooth<T>& a, const Frame<TL, TL + 6>& F, T* X, T* B, T* R, T* D0,
                                               T* D1, const T* sW, const T* sD, const T* sM, const T* x_in,
                                               const T* xc, const T* b, T* x_out, T* mx_out, TO* out, T oscale) {
  constexpr int S = TL + 6;
  // all global loads of this thread first (in flight together), then the stores
  constexpr int NL = (S * S + TILE_THREADS - 1) / TILE_THREADS;
  T xr[NL], br[NL];
#pragma unroll
  for (int k = 0; k < NL; ++k) {
    const int t = threadIdx.x + k * TILE_THREADS;
    Vtx<2> v;
    xr[k] = (T)0;
    br[k] = (T)0;
    if (t < S * S && tile_vertex<TL, S, INT>(F, t % S, t / S, v)) {
      const long long gi = gidx(F, v);
      br[k] = b[gi];
      const T xv = x_in[gi];
      // prolongation, as prolong_add_at
      const long long ci = (long long)(v.p[0] >> 1) + a.gc.sy * (v.p[1] >> 1);
      const long long cj = (long long)((v.p[0] >> 1) + (v.p[0] & 1)) + a.gc.sy * ((v.p[1] >> 1) + (v.p[1] & 1));
      const bool mid = (v.p[0] & 1) || (v.p[1] & 1);
      const T xci = xc[ci], xcj = xc[cj];
      xr[k] = mid ? fma((T)0.5, xci + xcj, xv) : xv + xci;
    }
  }
#pragma unroll
  for (int k = 0; k < NL; ++k) {
    const int t = threadIdx.x + k * TILE_THREADS;
    if (t < S * S) {
      X[t] = xr[k];
      B[t] = br[k];
    }
  }
  __syncthreads();
  const Geom& lg = F.lg;
  const RegW<2, T> rw = reg_weights<2, T>(sW, sD, 4);   // interior class, used when INT
  tile_loop<TL, S, 1, S - 1, INT>(F, [&](const Vtx<2>& v) {
    if constexpr (INT) resid_init_r<2, T>(lg, v, rw, B, X, R, D0, a.inv_th);
    else resid_init_at<2, T>(lg, v, sW, sD, B, X, R, D0, a.inv_th);
  });
  tile_loop<TL, S, 2, S - 2, INT>(F, [&](const Vtx<2>& v) {
    if constexpr (INT) cheb_step_r<2, T>(lg, v, rw, X, R, D0, D1, a.c1, a.c2, false);
    else cheb_step_at<2, T>(lg, v, sW, sD, X, R, D0, D1, a.c1, a.c2, false);
  });
  tile_loop<TL, S, 2, S - 2, INT>(F, [&](const Vtx<2>& v) {
    if constexpr (INT) cheb_last_r<2, T>(lg, v, rw, X, (T*)nullptr, D1, false);
    else cheb_last_at<2, T, T>(lg, v, sW, X, (T*)nullptr, D1, false, (T*)nullptr, (T)1);
  });
  tile_loop<TL, S, Frame<TL, S>::H, Frame<TL, S>::H + TL, INT>(F, [&](const Vtx<2>& v) {
    const long long gi = gidx(F, v);
    x_out[gi] = X[v.idx];
    if (out) out[gi] = (TO)(X[v.idx] * oscale);
    if (mx_out) {
      T xs[Topo<2>::NOFF];
      load_nb<2>(X, lg, v, xs);
      T acc = dot_w<2, Topo<2>::NOFF>(sM, v.cls, xs);
      acc *= (T)1;
      mx_out[gi] = acc;
    }
  });
}

template <typename T, typename TO, int TL>
__global__ void __launch_bounds__(TILE_THREADS) k_tile_post(TileSmooth<T> a, const T* __restrict__ x_in,
                                                            const T* __restrict__ xc, const T* __restrict__ b,
                                                            T* __restrict__ x_out, T* __restrict__ mx_out,
                                                            TO* __restrict__ out, T oscale) {
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int S = TL + 6, SS = S * S;
  const Frame<TL, S> F = make_frame<TL, S>(a.g);
  T* X = reinterpret_cast<T*>(smraw);
  T* B = X + SS;
  T* R = B + SS;
  T* D0 = R + SS;
  T* D1 = D0 + SS;
  T* sW = D1 + SS;
  T* sD = sW + Topo<2>::NCLASS * Topo<2>::NOFF;
  T* sM = sD + Topo<2>::NCLASS;
  load_tables<T>(sW, sD, a.W, a.dinv);
  if (mx_out)
    for (int i = threadIdx.x; i < Topo<2>::NCLASS * Topo<2>::NOFF; i += TILE_THREADS) sM[i] = a.WM[i];
  if (tile_interior(F)) tile_post_body<T, TO, TL, true>(a, F, X, B, R, D0, D1, sW, sD, sM, x_in, xc, b, x_out, mx_out, out, oscale);
  else tile_post_body<T, TO, TL, false>(a, F, X, B, R, D0, D1, sW, sD, sM, x_in, xc, b, x_out, mx_out, out, oscale);
}

// ---------------------------------------------------------------------------
// QTILE Chebyshev steps on M + C-step:  z1 = A~^{-1} r1,  t = r2 - C z1
// ---------------------------------------------------------------------------
template <typename T, typename TZ, bool INT>
__device__ __forceinline__ void tile_amass_body(const TileMass<T>& a, const Frame<TILE, TILE + 2 * QTILE>& F, T* X, T* B,
                                                T* R, T* D0, T* D1, const T* sW, const T* sD, const double* v,
                                                TZ* z1, T* t_out) {
  constexpr int S = TILE + 2 * QTILE, Q = QTILE;
  // all global loads of this thread first (in flight together), then the stores
  constexpr int NL = (S * S + TILE_THREADS - 1) / TILE_THREADS;
  double br[NL];
#pragma unroll
  for (int k = 0; k < NL; ++k) {
    const int t = threadIdx.x + k * TILE_THREADS;
    Vtx<2> vv;
    br[k] = 0.0;
    if (t < S * S && tile_vertex<TILE, S, INT>(F, t % S, t / S, vv)) br[k] = v[gidx(F, vv)];
  }
#pragma unroll
  for (int k = 0; k < NL; ++k) {
    const int t = threadIdx.x + k * TILE_THREADS;
    if (t < S * S) {
      X[t] = (T)0;
      B[t] = (T)br[k];
    }
  }
  __syncthreads();
  const Geom& lg = F.lg;
  const RegW<2, T> rw = reg_weights<2, T>(sW, sD, 4);   // interior class, used when INT
  tile_loop<TILE, S, 0, S, INT>(F, [&](const Vtx<2>& w) {
    if constexpr (INT) cheb_init_r<2, T>(w, rw, B, R, D0, a.inv_th);
    else cheb_init_at<2, T, T>(w, sD, B, (T)1, R, D0, a.inv_th);
  });
  T* Dd[2] = {D0, D1};
  static_for<0, Q - 1>([&](auto Kc) {
    constexpr int k = decltype(Kc)::value;
    T* din = Dd[k & 1];
    T* dout = Dd[(k + 1) & 1];
    tile_loop<TILE, S, k + 1, S - k - 1, INT>(F, [&](const Vtx<2>& w) {
      if constexpr (INT) cheb_step_r<2, T>(lg, w, rw, X, R, din, dout, a.c1[k], a.c2[k], k == 0);
      else cheb_step_at<2, T>(lg, w, sW, sD, X, R, din, dout, a.c1[k], a.c2[k], k == 0);
    });
  });
  T* dl = Dd[(Q - 1) & 1];
  tile_loop<TILE, S, Q - 1, S - Q + 1, INT>(F, [&](const Vtx<2>& w) {
    if constexpr (INT) cheb_last_r<2, T>(lg, w, rw, X, (T*)nullptr, dl, Q == 1);
    else cheb_last_at<2, T, T>(lg, w, sW, X, (T*)nullptr, dl, Q == 1, (T*)nullptr, (T)1);
  });
  const long long nv = a.g.nv;
  tile_loop<TILE, S, Q, Q + TILE, INT>(F, [&](const Vtx<2>& w) {
    const long long gi = gidx(F, w);
    z1[gi] = (TZ)(X[w.idx] * a.inv_a11);
    // C (inv_a11 X), as capply_at: self first, then +pos / -pos pairs
    T acc = a.coef[gi] * X[w.idx] * a.inv_a11;
    static_for<0, Topo<2>::NPOS>([&](auto P) {
      constexpr int p = decltype(P)::value;
      constexpr int op = 2 * p + 1, om = 2 * p + 2;
      if (nb_valid<2, op>(w.c))
        acc = fma(a.coef[(1 + p) * nv + gi], X[w.idx + nb_delta<2, op>(lg)] * a.inv_a11, acc);
      if (nb_valid<2, om>(w.c))
        acc = fma(a.coef[(1 + p) * nv + gi + nb_delta<2, om>(a.g)], X[w.idx + nb_delta<2, om>(lg)] * a.inv_a11, acc);
    });
    t_out[gi] = (T)v[gi + nv] * (T)1 - acc;
  });
}

template <typename T, typename TZ>
__global__ void __launch_bounds__(TILE_THREADS) k_tile_amass(TileMass<T> a, const double* __restrict__ v,
                                                             TZ* __restrict__ z1, T* __restrict__ t_out) {
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int S = TILE + 2 * QTILE, SS = S * S;
  const Frame<TILE, S> F = make_frame<TILE, S>(a.g);
  T* X = reinterpret_cast<T*>(smraw);
  T* B = X + SS;
  T* R = B + SS;
  T* D0 = R + SS;
  T* D1 = D0 + SS;
  T* sW = D1 + SS;
  T* sD = sW + Topo<2>::NCLASS * Topo<2>::NOFF;
  load_tables<T>(sW, sD, a.WM, a.dinvM);
  if (tile_interior(F)) tile_amass_body<T, TZ, true>(a, F, X, B, R, D0, D1, sW, sD, v, z1, t_out);
  else tile_amass_body<T, TZ, false>(a, F, X, B, R, D0, D1, sW, sD, v, z1, t_out);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static inline dim3 tile_grid(const Geom& g, int tl) {
  const int nb = (g.n1 + tl - 1) / tl;
  return dim3(nb, nb, 1);
}
static inline size_t tile_smem(int tl, int H, size_t elem) {
  const size_t S = tl + 2 * H;
  return (5 * S * S + 2 * Topo<2>::NCLASS * Topo<2>::NOFF + Topo<2>::NCLASS) * elem;
}

template <typename T>
void launch_tile_pre(const TileSmooth<T>& a, const T* x_in, const T* b, T* x_out, T* bc, cudaStream_t s) {
  if (a.tile == 16)
    count_launch(), k_tile_pre<T, 16><<<tile_grid(a.g, 16), TILE_THREADS, tile_smem(16, 4, sizeof(T)), s>>>(
                        a, x_in, b, x_out, bc);
  else
    count_launch(), k_tile_pre<T, 32><<<tile_grid(a.g, 32), TILE_THREADS, tile_smem(32, 4, sizeof(T)), s>>>(
                        a, x_in, b, x_out, bc);
}
template <typename T, typename TO>
void launch_tile_post(const TileSmooth<T>& a, const T* x_in, const T* xc, const T* b, T* x_out, T* mx_out, TO* out,
                      T oscale, cudaStream_t s) {
  if (a.tile == 16)
    count_launch(), k_tile_post<T, TO, 16><<<tile_grid(a.g, 16), TILE_THREADS, tile_smem(16, 3, sizeof(T)), s>>>(
                        a, x_in, xc, b, x_out, mx_out, out, oscale);
  else
    count_launch(), k_tile_post<T, TO, 32><<<tile_grid(a.g, 32), TILE_THREADS, tile_smem(32, 3, sizeof(T)), s>>>(
                        a, x_in, xc, b, x_out, mx_out, out, oscale);
}
template <typename T, typename TZ>
void launch_tile_amass(const TileMass<T>& a, const double* v, TZ* z1, T* t_out, cudaStream_t s) {
  count_launch(), k_tile_amass<T, TZ><<<tile_grid(a.g, TILE), TILE_THREADS, tile_smem(TILE, QTILE, sizeof(T)), s>>>(
                      a, v, z1, t_out);
}

template <typename T>
cudaError_t prepare_tiles(int q) {
  (void)q;
  const cudaFuncAttribute attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(k_tile_pre<T, 32>, attr, (int)tile_smem(32, 4, sizeof(T)));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tile_pre<T, 16>, attr, (int)tile_smem(16, 4, sizeof(T)));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tile_post<T, float, 32>, attr, (int)tile_smem(32, 3, sizeof(T)));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tile_post<T, double, 32>, attr, (int)tile_smem(32, 3, sizeof(T)));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tile_post<T, float, 16>, attr, (int)tile_smem(16, 3, sizeof(T)));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tile_post<T, double, 16>, attr, (int)tile_smem(16, 3, sizeof(T)));
  const int c = (int)tile_smem(TILE, QTILE, sizeof(T));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tile_amass<T, float>, attr, c);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tile_amass<T, double>, attr, c);
  return e;
}

#define OK_TILE_INST(T)                                                                                       \
  template void launch_tile_pre<T>(const TileSmooth<T>&, const T*, const T*, T*, T*, cudaStream_t);           \
  template void launch_tile_post<T, T>(const TileSmooth<T>&, const T*, const T*, const T*, T*, T*, T*, T,     \
                                       cudaStream_t);                                                         \
  template void launch_tile_amass<T, T>(const TileMass<T>&, const double*, T*, T*, cudaStream_t);             \
  template cudaError_t prepare_tiles<T>(int);
OK_TILE_INST(float)
OK_TILE_INST(double)
template void launch_tile_post<float, double>(const TileSmooth<float>&, const float*, const float*, const float*,
                                              float*, float*, double*, float, cudaStream_t);
template void launch_tile_post<double, float>(const TileSmooth<double>&, const double*, const double*,
                                              const double*, double*, double*, float*, double, cudaStream_t);
template void launch_tile_amass<float, double>(const TileMass<float>&, const double*, double*, float*, cudaStream_t);
template void launch_tile_amass<double, float>(const TileMass<double>&, const double*, float*, double*,
                                               cudaStream_t);

}  // namespace okg
