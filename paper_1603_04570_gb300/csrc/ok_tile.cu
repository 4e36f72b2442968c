// ok_tile.cu -- register-strip kernels with temporal blocking (2D grids).
//
// One thread block computes a CW x CH window of vertices of one multigrid
// level: the (CW - 2H) x (CH - 2H) vertices it owns and a halo of H on each
// side, so that H dependent stencil steps run without a grid-wide
// synchronisation (the halo is recomputed by the neighbouring blocks instead
// of exchanged).  Thread (column lx, chunk ty) holds the RY vertices
// lx x [ty RY, ty RY + RY) of every state vector in registers; before each
// stencil step it writes its own values into a shared-memory exchange buffer
// (two buffers, used alternately, so one barrier per step suffices) and reads
// back only what lies in the columns lx - 1 and lx + 1 and the two rows
// beyond its strip: 2 RY + 4 shared-memory reads and RY writes per RY
// vertices, the rest of the 7-point stencil comes from its own registers.
// Each step's result is garbage in one more ring of the window (the
// outermost ring reads the never-written pad of the exchange buffer); H is
// the number of dependent stencil steps, so the owned vertices stay exact.
//
// Every vertex update is the arithmetic of the per-vertex bodies of
// ok_stencil.cuh in the same order, so results are bitwise those of the
// one-kernel-per-step path.
//
//   k_strip_pre   two Chebyshev--Jacobi pre-smoothing steps on S_hat from x
//                 (or from zero), the residual, and its restriction P^T r to
//                 the coarser level (H = 4);
//   k_strip_post  prolongation x += P x_c and two post-smoothing steps, then
//                 optionally M x (the middle factor of
//                 S~^{-1} = S_hat^{-1} M S_hat^{-1}) and a cast of x (H = 3);
//   k_strip_amass QTILE Chebyshev steps on M (A~^{-1} r1, Sec. 3) and the
//                 preconditioner's C-step t = r2 - C A~^{-1} r1 (eqn prec),
//                 in two launches of halo QSPLIT.
// x is read from one buffer and written to another (ping-pong), because other
// blocks read the old x in their halos while this block writes.
#include "ok_internal.cuh"
#include "ok_kernels.h"
#include "ok_stencil.cuh"

namespace okg {

constexpr int QTILE = 10;   // mass Chebyshev steps handled by the strip kernels
constexpr int QSPLIT = 5;   // steps of the first of the two mass launches
constexpr int NTAB = Topo<2>::NCLASS * Topo<2>::NOFF;

// Window geometry: CW columns, CH = RY * NCH rows, halo H.
template <int CW_, int RY_, int NCH_, int H_> struct SG {
  static constexpr int CW = CW_, RY = RY_, NCH = NCH_, H = H_;
  static constexpr int CH = RY * NCH;
  static constexpr int OW = CW - 2 * H, OH = CH - 2 * H;   // owned extents
  static constexpr int SW = CW + 2;                        // exchange row stride (pad column each side)
  static constexpr int SB = (CH + 2) * SW;                 // one exchange buffer (pad row above and below)
  static constexpr int NT = CW * NCH;                      // threads
  static_assert(OW > 0 && OH > 0, "halo too wide for the window");
  static_assert(CW % 32 == 0, "a warp covers 32 consecutive columns of one chunk");
};

// window sizes (CW, RY, NCH) per precision: large levels, small levels, the
// mass kernel; each may be set at compile time
// (measured on the 1025^2 hierarchy: short strips and many threads win, the
// kernels being latency- rather than throughput-bound)
#ifndef OK_STRIP_F_BIG
#define OK_STRIP_F_BIG 64, 8, 4
#endif
#ifndef OK_STRIP_F_SMALL
#define OK_STRIP_F_SMALL 32, 2, 16
#endif
#ifndef OK_STRIP_F_MASS
#define OK_STRIP_F_MASS 64, 4, 16
#endif
template <typename T> struct StripCfg;
template <> struct StripCfg<float> {
  template <int H> using Big = SG<OK_STRIP_F_BIG, H>;
  template <int H> using Small = SG<OK_STRIP_F_SMALL, H>;
  // further shapes the autotuner may pick per level (shape ids 2, 3, 4)
  template <int H> using S2 = SG<64, 4, 8, H>;
  template <int H> using S3 = SG<64, 4, 16, H>;
  template <int H> using S4 = SG<128, 4, 8, H>;
  using Mass = SG<OK_STRIP_F_MASS, QSPLIT>;
  template <int H> using Low = SG<64, 4, 16, H>;       // one window per block of the cluster kernel
};
#ifndef OK_STRIP_D_BIG
#define OK_STRIP_D_BIG 64, 2, 16
#endif
#ifndef OK_STRIP_D_SMALL
#define OK_STRIP_D_SMALL 32, 2, 8
#endif
#ifndef OK_STRIP_D_MASS
#define OK_STRIP_D_MASS 64, 2, 16
#endif
template <> struct StripCfg<double> {
  template <int H> using Big = SG<OK_STRIP_D_BIG, H>;
  template <int H> using Small = SG<OK_STRIP_D_SMALL, H>;
  template <int H> using S2 = SG<64, 4, 8, H>;
  template <int H> using S3 = SG<32, 4, 8, H>;
  template <int H> using S4 = SG<64, 2, 8, H>;
  using Mass = SG<OK_STRIP_D_MASS, QSPLIT>;
  template <int H> using Low = SG<64, 2, 16, H>;
};

// this thread's strip
struct Pos {
  int lx, ly0;     // local column, first local row
  int gx, gy0;     // global coordinates of (lx, ly0)
  int cx;          // axis class of the column
  bool colin;      // 0 <= gx <= n
};

// window (wx, wy) of a level: owned vertices [wx OW, wx OW + OW) x [wy OH, wy OH + OH)
template <class G>
__device__ __forceinline__ Pos strip_pos(int n, int wx, int wy) {
  Pos p;
  p.lx = threadIdx.x % G::CW;
  p.ly0 = (threadIdx.x / G::CW) * G::RY;
  p.gx = wx * G::OW - G::H + p.lx;
  p.gy0 = wy * G::OH - G::H + p.ly0;
  p.colin = p.gx >= 0 && p.gx <= n;
  p.cx = axis_class(p.gx, n);
  return p;
}

// every vertex of the window strictly inside the domain (interior class)?
template <class G>
__device__ __forceinline__ bool strip_interior(int n, int wx, int wy) {
  const int x0 = wx * G::OW - G::H, y0 = wy * G::OH - G::H;
  return x0 >= 1 && y0 >= 1 && x0 + G::CW - 1 <= n - 1 && y0 + G::CH - 1 <= n - 1;
}

// Global load of data that other thread blocks of the same launch may have
// written (CG: through L2, never a stale L1 line or the read-only path).
template <bool CG, typename T>
__device__ __forceinline__ T ldg(const T* p) {
  if constexpr (CG) return __ldcg(p);
  else return *p;
}

__device__ __forceinline__ bool row_in(const Pos& p, int i, int n) {
  const int gy = p.gy0 + i;
  return p.colin && gy >= 0 && gy <= n;
}
template <class G>
__device__ __forceinline__ bool owned(const Pos& p, int i) {
  const int ly = p.ly0 + i;
  return p.lx >= G::H && p.lx < G::CW - G::H && ly >= G::H && ly < G::CH - G::H;
}

// ---- exchange of one state vector through shared memory -------------------
template <class G, typename T>
__device__ __forceinline__ void xput(T* buf, const Pos& p, const T (&v)[G::RY]) {
#pragma unroll
  for (int i = 0; i < G::RY; ++i) buf[(p.ly0 + i + 1) * G::SW + p.lx + 1] = v[i];
}

template <class G, typename T> struct Nb {
  T dn, up;              // own column, rows ly0 - 1 and ly0 + RY
  T L[G::RY + 1];        // column lx - 1, rows ly0 - 1 .. ly0 + RY - 1
  T R[G::RY + 1];        // column lx + 1, rows ly0 .. ly0 + RY
};

template <class G, typename T>
__device__ __forceinline__ void xget(const T* buf, const Pos& p, Nb<G, T>& nb) {
  const T* c = buf + p.ly0 * G::SW + p.lx + 1;     // own column, local row ly0 - 1
  nb.dn = c[0];
  nb.up = c[(G::RY + 1) * G::SW];
#pragma unroll
  for (int j = 0; j <= G::RY; ++j) {
    nb.L[j] = c[j * G::SW - 1];
    nb.R[j] = c[(j + 1) * G::SW + 1];
  }
}

// the 7 stencil values of row i in offset order (self, +x, -x, +y, -y, +xy,
// -xy), zero outside the domain as load_nb gives them
template <class G, typename T, bool INT>
__device__ __forceinline__ void nb_row(const T (&v)[G::RY], const Nb<G, T>& nb, int i, int cx, int cy,
                                       T (&xs)[Topo<2>::NOFF]) {
  xs[0] = v[i];
  xs[1] = nb.R[i];
  xs[2] = nb.L[i + 1];
  xs[3] = i + 1 < G::RY ? v[i + 1] : nb.up;
  xs[4] = i > 0 ? v[i - 1] : nb.dn;
  xs[5] = nb.R[i + 1];
  xs[6] = nb.L[i];
  if constexpr (!INT) {
    const int c[3] = {cx, cy, 1};
    static_for<1, Topo<2>::NOFF>([&](auto O) {
      constexpr int o = decltype(O)::value;
      if (!nb_valid<2, o>(c)) xs[o] = (T)0;
    });
  }
}

template <typename T, bool INT>
__device__ __forceinline__ T sdot(const RegW<2, T>& rw, const T* sW, int cls, const T (&xs)[Topo<2>::NOFF]) {
  if constexpr (INT) return dot_r<2, T>(rw, xs);
  else return dot_w<2, Topo<2>::NOFF>(sW, cls, xs);
}

template <bool INT>
__device__ __forceinline__ int row_class(const Pos& p, int i, int n, int& cy) {
  cy = INT ? 1 : axis_class(p.gy0 + i, n);
  return INT ? 4 : p.cx + 3 * cy;
}

template <typename T>
__device__ __forceinline__ void load_table(T* s, const T* g, int count, int nt) {
  for (int i = threadIdx.x; i < count; i += nt) s[i] = g[i];
}

// ---------------------------------------------------------------------------
// pre-smoothing (2 steps) + restriction
// ---------------------------------------------------------------------------
template <typename T, class G, bool INT, bool CG = false>
__device__ __forceinline__ void strip_pre_body(const TileSmooth<T>& a, const Pos& p, T* buf0, T* buf1,
                                               const T* sW, const T* sD, const T* x_in, const T* b, T* x_out,
                                               T* bc) {
  constexpr int RY = G::RY;
  const int n = a.g.n;
  const long long sy = a.g.sy;
  const bool xz = (x_in == nullptr);
  T bb[RY], x[RY], r[RY], d[RY];
#pragma unroll
  for (int i = 0; i < RY; ++i) {
    const bool in = INT || row_in(p, i, n);
    const long long gi = p.gx + sy * (p.gy0 + i);
    bb[i] = in ? ldg<CG>(b + gi) : (T)0;
    x[i] = (in && !xz) ? ldg<CG>(x_in + gi) : (T)0;
  }
  if (!xz) xput<G>(buf0, p, x);
  __syncthreads();                                  // tables (and x) visible
  RegW<2, T> rw{};
  if constexpr (INT) rw = reg_weights<2, T>(sW, sD, 4);
  Nb<G, T> nb;
  if (xz) {
#pragma unroll
    for (int i = 0; i < RY; ++i) {                  // cheb_init
      int cy;
      const int cls = row_class<INT>(p, i, n, cy);
      const T dv = INT ? rw.dinv : sD[cls];
      T rr = bb[i] * (T)1;
      r[i] = rr;
      d[i] = dv * rr * a.inv_th;
    }
  } else {
    xget<G>(buf0, p, nb);
#pragma unroll
    for (int i = 0; i < RY; ++i) {                  // resid_init
      int cy;
      const int cls = row_class<INT>(p, i, n, cy);
      const T dv = INT ? rw.dinv : sD[cls];
      T xs[Topo<2>::NOFF];
      nb_row<G, T, INT>(x, nb, i, p.cx, cy, xs);
      T rr = bb[i] - sdot<T, INT>(rw, sW, cls, xs);
      r[i] = rr;
      d[i] = dv * rr * a.inv_th;
    }
  }
  // first smoothing step (cheb_step, first when x started from zero)
  T dn[RY];
  xput<G>(buf1, p, d);
  __syncthreads();
  xget<G>(buf1, p, nb);
#pragma unroll
  for (int i = 0; i < RY; ++i) {
    int cy;
    const int cls = row_class<INT>(p, i, n, cy);
    const T dv = INT ? rw.dinv : sD[cls];
    T xs[Topo<2>::NOFF];
    nb_row<G, T, INT>(d, nb, i, p.cx, cy, xs);
    x[i] = (xz ? (T)0 : x[i]) + xs[0];
    T rr = r[i] - sdot<T, INT>(rw, sW, cls, xs);
    r[i] = rr;
    dn[i] = fma(a.c1, xs[0], a.c2 * (dv * rr));
  }
  // last smoothing step, keeping the residual (cheb_last with r)
  xput<G>(buf0, p, dn);
  __syncthreads();
  xget<G>(buf0, p, nb);
#pragma unroll
  for (int i = 0; i < RY; ++i) {
    int cy;
    const int cls = row_class<INT>(p, i, n, cy);
    T xs[Topo<2>::NOFF];
    nb_row<G, T, INT>(dn, nb, i, p.cx, cy, xs);
    T xx = x[i] + xs[0];
    r[i] = r[i] - sdot<T, INT>(rw, sW, cls, xs);
    x[i] = xx;
  }
  // restriction (restrict_at) at the coarse vertices whose fine centre this
  // block owns, and the owned part of x
  xput<G>(buf1, p, r);
  __syncthreads();
  xget<G>(buf1, p, nb);
  const long long scy = a.gc.sy;
#pragma unroll
  for (int i = 0; i < RY; ++i) {
    const int gy = p.gy0 + i;
    if (!owned<G>(p, i) || !(INT || row_in(p, i, n))) continue;
    x_out[p.gx + sy * gy] = x[i];
    if ((p.gx & 1) || (gy & 1)) continue;
    int cy;
    row_class<INT>(p, i, n, cy);
    T xs[Topo<2>::NOFF];
    nb_row<G, T, INT>(r, nb, i, p.cx, cy, xs);
    T acc = (T)0;
#pragma unroll
    for (int o = 1; o < Topo<2>::NOFF; ++o) acc += xs[o];     // zero where restrict_at skips
    bc[(p.gx >> 1) + scy * (gy >> 1)] = fma((T)0.5, acc, xs[0]);
  }
}

template <typename T, class G>
__device__ __forceinline__ void strip_pre_kernel(const TileSmooth<T>& a, const T* __restrict__ x_in,
                                                 const T* __restrict__ b, T* __restrict__ x_out,
                                                 T* __restrict__ bc) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* buf0 = reinterpret_cast<T*>(smraw);
  T* buf1 = buf0 + G::SB;
  T* sW = buf1 + G::SB;
  T* sD = sW + NTAB;
  load_table<T>(sW, a.W, NTAB, G::NT);
  load_table<T>(sD, a.dinv, Topo<2>::NCLASS, G::NT);
  pdl_wait();                                      // tables are fixed at setup; the rest is not
  const Pos p = strip_pos<G>(a.g.n, blockIdx.x, blockIdx.y);
  if (strip_interior<G>(a.g.n, blockIdx.x, blockIdx.y))
    strip_pre_body<T, G, true>(a, p, buf0, buf1, sW, sD, x_in, b, x_out, bc);
  else
    strip_pre_body<T, G, false>(a, p, buf0, buf1, sW, sD, x_in, b, x_out, bc);
}
template <typename T, class G>
__global__ void __launch_bounds__(G::NT) k_strip_pre(TileSmooth<T> a, const T* __restrict__ x_in,
                                                      const T* __restrict__ b, T* __restrict__ x_out,
                                                      T* __restrict__ bc) {
  pdl_launch_dependents();
  strip_pre_kernel<T, G>(a, x_in, b, x_out, bc);
}
template <typename T, class G>
__global__ void __launch_bounds__(G::NT) k_strip_pre_b(Batch<StripPreItem<T>> B) {
  pdl_launch_dependents();
  const StripPreItem<T>& it = B.a[blockIdx.z];
  strip_pre_kernel<T, G>(it.a, it.x_in, it.b, it.x_out, it.bc);
}

// ---------------------------------------------------------------------------
// prolongation + post-smoothing (2 steps) [+ M x] [+ cast of x]
// ---------------------------------------------------------------------------
template <typename T, typename TO, class G, bool INT, bool CG = false>
__device__ __forceinline__ void strip_post_body(const TileSmooth<T>& a, const Pos& p, T* buf0, T* buf1,
                                                const T* sW, const T* sD, const T* sM, const T* x_in,
                                                const T* xc, const T* b, T* x_out, T* mx_out, TO* out,
                                                T oscale) {
  constexpr int RY = G::RY;
  const int n = a.g.n;
  const long long sy = a.g.sy, scy = a.gc.sy;
  T bb[RY], x[RY], r[RY], d[RY];
  const int hx = p.gx >> 1, ox = p.gx & 1;
#pragma unroll
  for (int i = 0; i < RY; ++i) {
    const bool in = INT || row_in(p, i, n);
    const int gy = p.gy0 + i;
    const long long gi = p.gx + sy * gy;
    bb[i] = (T)0;
    x[i] = (T)0;
    if (in) {
      bb[i] = ldg<CG>(b + gi);
      const T xv = ldg<CG>(x_in + gi);
      // prolongation, as prolong_add_at
      const int hy = gy >> 1, oy = gy & 1;
      const long long ci = (long long)hx + scy * hy;
      const long long cj = (long long)(hx + ox) + scy * (hy + oy);
      const bool mid = ox || oy;
      const T xci = ldg<CG>(xc + ci), xcj = ldg<CG>(xc + cj);
      x[i] = mid ? fma((T)0.5, xci + xcj, xv) : xv + xci;
    }
  }
  xput<G>(buf0, p, x);
  __syncthreads();                                  // tables and x visible
  RegW<2, T> rw{};
  if constexpr (INT) rw = reg_weights<2, T>(sW, sD, 4);
  Nb<G, T> nb;
  xget<G>(buf0, p, nb);
#pragma unroll
  for (int i = 0; i < RY; ++i) {                    // resid_init
    int cy;
    const int cls = row_class<INT>(p, i, n, cy);
    const T dv = INT ? rw.dinv : sD[cls];
    T xs[Topo<2>::NOFF];
    nb_row<G, T, INT>(x, nb, i, p.cx, cy, xs);
    T rr = bb[i] - sdot<T, INT>(rw, sW, cls, xs);
    r[i] = rr;
    d[i] = dv * rr * a.inv_th;
  }
  T dn[RY];
  xput<G>(buf1, p, d);
  __syncthreads();
  xget<G>(buf1, p, nb);
#pragma unroll
  for (int i = 0; i < RY; ++i) {                    // cheb_step (not first)
    int cy;
    const int cls = row_class<INT>(p, i, n, cy);
    const T dv = INT ? rw.dinv : sD[cls];
    T xs[Topo<2>::NOFF];
    nb_row<G, T, INT>(d, nb, i, p.cx, cy, xs);
    x[i] = x[i] + xs[0];
    T rr = r[i] - sdot<T, INT>(rw, sW, cls, xs);
    r[i] = rr;
    dn[i] = fma(a.c1, xs[0], a.c2 * (dv * rr));
  }
#pragma unroll
  for (int i = 0; i < RY; ++i) {                    // cheb_last without the residual
    T xx = x[i] + dn[i];
    x[i] = xx;
  }
#pragma unroll
  for (int i = 0; i < RY; ++i) {
    if (!owned<G>(p, i) || !(INT || row_in(p, i, n))) continue;
    const long long gi = p.gx + sy * (p.gy0 + i);
    x_out[gi] = x[i];
    if (out) out[gi] = (TO)(x[i] * oscale);
  }
  if (mx_out) {                                     // M x (op_apply with alpha = 1)
    xput<G>(buf0, p, x);
    __syncthreads();
    xget<G>(buf0, p, nb);
#pragma unroll
    for (int i = 0; i < RY; ++i) {
      if (!owned<G>(p, i) || !(INT || row_in(p, i, n))) continue;
      int cy;
      const int cls = row_class<INT>(p, i, n, cy);
      T xs[Topo<2>::NOFF];
      nb_row<G, T, INT>(x, nb, i, p.cx, cy, xs);
      T acc = dot_w<2, Topo<2>::NOFF>(sM, cls, xs);
      acc *= (T)1;
      mx_out[p.gx + sy * (p.gy0 + i)] = acc;
    }
  }
}

template <typename T, typename TO, class G>
__device__ __forceinline__ void strip_post_kernel(const TileSmooth<T>& a, const T* __restrict__ x_in,
                                                  const T* __restrict__ xc, const T* __restrict__ b,
                                                  T* __restrict__ x_out, T* __restrict__ mx_out,
                                                  TO* __restrict__ out, T oscale) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* buf0 = reinterpret_cast<T*>(smraw);
  T* buf1 = buf0 + G::SB;
  T* sW = buf1 + G::SB;
  T* sD = sW + NTAB;
  T* sM = sD + Topo<2>::NCLASS;
  load_table<T>(sW, a.W, NTAB, G::NT);
  load_table<T>(sD, a.dinv, Topo<2>::NCLASS, G::NT);
  if (mx_out) load_table<T>(sM, a.WM, NTAB, G::NT);
  pdl_wait();                                      // tables are fixed at setup; the rest is not
  const Pos p = strip_pos<G>(a.g.n, blockIdx.x, blockIdx.y);
  if (strip_interior<G>(a.g.n, blockIdx.x, blockIdx.y))
    strip_post_body<T, TO, G, true>(a, p, buf0, buf1, sW, sD, sM, x_in, xc, b, x_out, mx_out, out, oscale);
  else
    strip_post_body<T, TO, G, false>(a, p, buf0, buf1, sW, sD, sM, x_in, xc, b, x_out, mx_out, out, oscale);
}
template <typename T, typename TO, class G>
__global__ void __launch_bounds__(G::NT) k_strip_post(TileSmooth<T> a, const T* __restrict__ x_in,
                                                       const T* __restrict__ xc, const T* __restrict__ b,
                                                       T* __restrict__ x_out, T* __restrict__ mx_out,
                                                       TO* __restrict__ out, T oscale) {
  pdl_launch_dependents();
  strip_post_kernel<T, TO, G>(a, x_in, xc, b, x_out, mx_out, out, oscale);
}
template <typename T, typename TO, class G>
__global__ void __launch_bounds__(G::NT) k_strip_post_b(Batch<StripPostItem<T, TO>> B) {
  pdl_launch_dependents();
  const StripPostItem<T, TO>& it = B.a[blockIdx.z];
  strip_post_kernel<T, TO, G>(it.a, it.x_in, it.xc, it.b, it.x_out, it.mx_out, it.out, it.oscale);
}

// ---------------------------------------------------------------------------
// QTILE Chebyshev steps on M + C-step:  z1 = A~^{-1} r1,  t = r2 - C z1, in
// two launches of QSPLIT and QTILE - 1 - QSPLIT steps (halo 5 each instead of
// 10 in one: a third less redundant work); the first stores x, r, d of its
// owned vertices for the second, whose windows reload them with their halo.
// ---------------------------------------------------------------------------
template <typename T, typename TZ, class G, bool INT, int K0, int K1, bool FIRST, bool LAST>
__device__ __forceinline__ void strip_amass_body(const TileMass<T>& a, const Pos& p, T* buf0, T* buf1,
                                                 const T* sW, const T* sD, const double* v, TZ* z1, T* t_out) {
  static_assert(G::H >= (K1 - K0) + (LAST ? 1 : 0), "halo too narrow for the steps of this launch");
  constexpr int RY = G::RY, Q = QTILE;
  const int n = a.g.n;
  const long long sy = a.g.sy, nv = a.g.nv;
  T x[RY], r[RY], d[RY];
#pragma unroll
  for (int i = 0; i < RY; ++i) {
    const bool in = INT || row_in(p, i, n);
    const long long gi = p.gx + sy * (p.gy0 + i);
    if constexpr (FIRST) {
      x[i] = (T)0;
      r[i] = in ? (T)v[gi] : (T)0;                  // b, held until the tables arrive
    } else {
      x[i] = in ? a.sx[gi] : (T)0;
      r[i] = in ? a.sr[gi] : (T)0;
      d[i] = in ? a.sd[gi] : (T)0;
    }
  }
  __syncthreads();                                  // tables visible
  RegW<2, T> rw{};
  if constexpr (INT) rw = reg_weights<2, T>(sW, sD, 4);
  if constexpr (FIRST) {
#pragma unroll
    for (int i = 0; i < RY; ++i) {                  // cheb_init (b scaled by 1)
      int cy;
      const int cls = row_class<INT>(p, i, n, cy);
      const T dv = INT ? rw.dinv : sD[cls];
      T rr = r[i] * (T)1;
      r[i] = rr;
      d[i] = dv * rr * a.inv_th;
    }
  }
  Nb<G, T> nb;
  static_for<K0, K1>([&](auto Kc) {                 // cheb_step k (first at k = 0)
    constexpr int k = decltype(Kc)::value;
    T* buf = ((k - K0) & 1) ? buf1 : buf0;
    xput<G>(buf, p, d);
    __syncthreads();
    xget<G>(buf, p, nb);
    T dn[RY];
#pragma unroll
    for (int i = 0; i < RY; ++i) {
      int cy;
      const int cls = row_class<INT>(p, i, n, cy);
      const T dv = INT ? rw.dinv : sD[cls];
      T xs[Topo<2>::NOFF];
      nb_row<G, T, INT>(d, nb, i, p.cx, cy, xs);
      x[i] = (k == 0 ? (T)0 : x[i]) + xs[0];
      T rr = r[i] - sdot<T, INT>(rw, sW, cls, xs);
      r[i] = rr;
      dn[i] = fma(a.c1[k], xs[0], a.c2[k] * (dv * rr));
    }
#pragma unroll
    for (int i = 0; i < RY; ++i) d[i] = dn[i];
  });
  if constexpr (!LAST) {                            // hand x, r, d of the owned vertices on
#pragma unroll
    for (int i = 0; i < RY; ++i) {
      if (!owned<G>(p, i) || !(INT || row_in(p, i, n))) continue;
      const long long gi = p.gx + sy * (p.gy0 + i);
      a.sx[gi] = x[i];
      a.sr[gi] = r[i];
      a.sd[gi] = d[i];
    }
    return;
  } else {
#pragma unroll
    for (int i = 0; i < RY; ++i) {                  // cheb_last without the residual
      T xx = (Q == 1 ? (T)0 : x[i]) + d[i];
      x[i] = xx;
    }
    // C-step at the owned vertices (capply_at on y = x, scaled by 1 / a11)
    T* buf = ((K1 - K0) & 1) ? buf1 : buf0;
    xput<G>(buf, p, x);
    __syncthreads();
    xget<G>(buf, p, nb);
#pragma unroll
    for (int i = 0; i < RY; ++i) {
      if (!owned<G>(p, i) || !(INT || row_in(p, i, n))) continue;
      const long long gi = p.gx + sy * (p.gy0 + i);
      int cy;
      row_class<INT>(p, i, n, cy);
      const int c[3] = {p.cx, cy, 1};
      z1[gi] = (TZ)(x[i] * a.inv_a11);
      T xs[Topo<2>::NOFF];
      nb_row<G, T, INT>(x, nb, i, p.cx, cy, xs);
      T acc = a.coef[gi] * xs[0] * a.inv_a11;
      static_for<0, Topo<2>::NPOS>([&](auto P) {
        constexpr int q = decltype(P)::value;
        constexpr int op = 2 * q + 1, om = 2 * q + 2;
        constexpr long long dxm = off_comp(2, om, 0), dym = off_comp(2, om, 1);
        if (INT || nb_valid<2, op>(c)) acc = fma(a.coef[(1 + q) * nv + gi], xs[op] * a.inv_a11, acc);
        if (INT || nb_valid<2, om>(c))
          acc = fma(a.coef[(1 + q) * nv + gi + dxm + sy * dym], xs[om] * a.inv_a11, acc);
      });
      t_out[gi] = (T)v[gi + nv] * (T)1 - acc;
    }
  }
}

template <typename T, typename TZ, class G, int K0, int K1, bool FIRST, bool LAST>
__device__ __forceinline__ void strip_amass_kernel(const TileMass<T>& a, const double* __restrict__ v,
                                                   TZ* __restrict__ z1, T* __restrict__ t_out) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* buf0 = reinterpret_cast<T*>(smraw);
  T* buf1 = buf0 + G::SB;
  T* sW = buf1 + G::SB;
  T* sD = sW + NTAB;
  load_table<T>(sW, a.WM, NTAB, G::NT);
  load_table<T>(sD, a.dinvM, Topo<2>::NCLASS, G::NT);
  pdl_wait();                                      // tables are fixed at setup; the rest is not
  const Pos p = strip_pos<G>(a.g.n, blockIdx.x, blockIdx.y);
  if (strip_interior<G>(a.g.n, blockIdx.x, blockIdx.y))
    strip_amass_body<T, TZ, G, true, K0, K1, FIRST, LAST>(a, p, buf0, buf1, sW, sD, v, z1, t_out);
  else
    strip_amass_body<T, TZ, G, false, K0, K1, FIRST, LAST>(a, p, buf0, buf1, sW, sD, v, z1, t_out);
}
template <typename T, typename TZ, class G, int K0, int K1, bool FIRST, bool LAST>
__global__ void __launch_bounds__(G::NT) k_strip_amass(TileMass<T> a, const double* __restrict__ v,
                                                        TZ* __restrict__ z1, T* __restrict__ t_out) {
  pdl_launch_dependents();
  strip_amass_kernel<T, TZ, G, K0, K1, FIRST, LAST>(a, v, z1, t_out);
}
template <typename T, typename TZ, class G, int K0, int K1, bool FIRST, bool LAST>
__global__ void __launch_bounds__(G::NT) k_strip_amass_b(Batch<AmassItem<T, TZ>> B) {
  pdl_launch_dependents();
  const AmassItem<T, TZ>& it = B.a[blockIdx.z];
  strip_amass_kernel<T, TZ, G, K0, K1, FIRST, LAST>(it.a, it.v, it.z1, it.t_out);
}

// ---------------------------------------------------------------------------
// bottom of the V-cycle in one cluster (see LowArgs in ok_kernels.h)
// ---------------------------------------------------------------------------
// all threads of all blocks of the cluster (every thread reaches every call:
// the phase loops are uniform); release/acquire at cluster scope orders the
// global-memory writes of one phase before the reads of the next.  The
// non-.aligned forms do not require the warp to be converged.
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

template <typename T, class GP, class GQ>
__global__ void __launch_bounds__(GP::NT, 1) k_low_vcycle(LowArgs<T> a) {
  static_assert(GP::NT == GQ::NT && GP::SB == GQ::SB, "pre and post windows share the block shape");
  pdl_entry();
  extern __shared__ __align__(16) unsigned char smraw[];
  T* buf0 = reinterpret_cast<T*>(smraw);
  T* buf1 = buf0 + GP::SB;
  T* sW = buf1 + GP::SB;
  T* sD = sW + NTAB;
  for (int i = 0; i < a.nl; ++i) {                  // pre-smoothing and restriction, finest first
    const TileSmooth<T>& ts = a.ts[i];
    const int nx = (ts.g.n1 + GP::OW - 1) / GP::OW, ny = (ts.g.n1 + GP::OH - 1) / GP::OH;
    for (int w = blockIdx.x; w < nx * ny; w += gridDim.x) {
      load_table<T>(sW, ts.W, NTAB, GP::NT);
      load_table<T>(sD, ts.dinv, Topo<2>::NCLASS, GP::NT);
      const int wx = w % nx, wy = w / nx;
      const Pos p = strip_pos<GP>(ts.g.n, wx, wy);
      if (strip_interior<GP>(ts.g.n, wx, wy))
        strip_pre_body<T, GP, true, true>(ts, p, buf0, buf1, sW, sD, (const T*)nullptr, a.rhs[i], a.P[i],
                                          a.rhs[i + 1]);
      else
        strip_pre_body<T, GP, false, true>(ts, p, buf0, buf1, sW, sD, (const T*)nullptr, a.rhs[i], a.P[i],
                                           a.rhs[i + 1]);
      __syncthreads();                              // exchange buffers and tables are reused
    }
    cluster_barrier();
  }
  {                                                 // coarsest level: xc = A rhs[nl]
    T* sb = buf0;
    gemv_stage_b<T, true>(a.nc, a.ldA, a.rhs[a.nl], sb);
    __syncthreads();
    constexpr int W = GP::NT / 32;
    for (long long r = (long long)blockIdx.x * W + (threadIdx.x >> 5); r < a.nc; r += (long long)gridDim.x * W) {
      const T v = gemv_row<T>(a.ldA, a.A, sb, r);
      if ((threadIdx.x & 31) == 0) a.xc[r] = v;
    }
  }
  cluster_barrier();
  for (int i = a.nl - 1; i >= 0; --i) {             // prolongation and post-smoothing, coarsest first
    const TileSmooth<T>& ts = a.ts[i];
    const T* xcoarse = i == a.nl - 1 ? a.xc : a.Q[i + 1];
    const int nx = (ts.g.n1 + GQ::OW - 1) / GQ::OW, ny = (ts.g.n1 + GQ::OH - 1) / GQ::OH;
    for (int w = blockIdx.x; w < nx * ny; w += gridDim.x) {
      load_table<T>(sW, ts.W, NTAB, GQ::NT);
      load_table<T>(sD, ts.dinv, Topo<2>::NCLASS, GQ::NT);
      const int wx = w % nx, wy = w / nx;
      const Pos p = strip_pos<GQ>(ts.g.n, wx, wy);
      if (strip_interior<GQ>(ts.g.n, wx, wy))
        strip_post_body<T, T, GQ, true, true>(ts, p, buf0, buf1, sW, sD, (const T*)nullptr, a.P[i], xcoarse,
                                              a.rhs[i], a.Q[i], (T*)nullptr, (T*)nullptr, (T)1);
      else
        strip_post_body<T, T, GQ, false, true>(ts, p, buf0, buf1, sW, sD, (const T*)nullptr, a.P[i], xcoarse,
                                               a.rhs[i], a.Q[i], (T*)nullptr, (T*)nullptr, (T)1);
      __syncthreads();
    }
    if (i > 0) cluster_barrier();
  }
}

template <typename T>
static size_t low_smem(long long nc) {
  using GP = typename StripCfg<T>::template Low<4>;
  const size_t win = (2 * (size_t)GP::SB + NTAB + Topo<2>::NCLASS) * sizeof(T);
  const size_t gem = (size_t)gemv_staged<T>(gemv_ld(nc, sizeof(T))) * sizeof(T);
  return win > gem ? win : gem;
}

template <typename T>
int prepare_low_vcycle(long long nc) {
  using GP = typename StripCfg<T>::template Low<4>;
  using GQ = typename StripCfg<T>::template Low<3>;
  auto kern = k_low_vcycle<T, GP, GQ>;
  (void)nc;
  const size_t smem = low_smem<T>(COARSE_NC_MAX);  // per-kernel limit shared by all handles
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  for (int c : {16, 8}) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(c, 1, 1);
    cfg.blockDim = dim3(GP::NT, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = c;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) == cudaSuccess && nclusters >= 1) return c;
    cudaGetLastError();
  }
  return 0;
}

template <typename T>
void launch_low_vcycle(const LowArgs<T>& a, int cluster, cudaStream_t s) {
  using GP = typename StripCfg<T>::template Low<4>;
  using GQ = typename StripCfg<T>::template Low<3>;
  count_launch();
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cluster, 1, 1);
  cfg.blockDim = dim3(GP::NT, 1, 1);
  cfg.dynamicSmemBytes = low_smem<T>(a.nc);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_low_vcycle<T, GP, GQ>, a);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <class G>
static inline dim3 strip_grid(const Geom& g) {
  return dim3((g.n1 + G::OW - 1) / G::OW, (g.n1 + G::OH - 1) / G::OH, 1);
}
template <class G, typename T>
static inline size_t strip_smem(bool with_m) {
  return (2 * (size_t)G::SB + NTAB + Topo<2>::NCLASS + (with_m ? NTAB : 0)) * sizeof(T);
}

// window shape `shape` (0: Small, 1: Big, 2..4: S2..S4) with halo H
template <typename T, int H, typename F>
static void with_shape(int shape, F&& f) {
  using C = StripCfg<T>;
  switch (shape) {
    case 1: f(typename C::template Big<H>{}); break;
    case 2: f(typename C::template S2<H>{}); break;
    case 3: f(typename C::template S3<H>{}); break;
    case 4: f(typename C::template S4<H>{}); break;
    default: f(typename C::template Small<H>{});
  }
}

template <typename T>
void launch_tile_pre(const TileSmooth<T>& a, const T* x_in, const T* b, T* x_out, T* bc, cudaStream_t s) {
  with_shape<T, 4>(a.tile, [&](auto G) {
    using GG = decltype(G);
    launch_k(k_strip_pre<T, GG>, strip_grid<GG>(a.g), GG::NT, strip_smem<GG, T>(false), s, a, x_in, b, x_out, bc);
  });
}
template <typename T, typename TO>
void launch_tile_post(const TileSmooth<T>& a, const T* x_in, const T* xc, const T* b, T* x_out, T* mx_out, TO* out,
                      T oscale, cudaStream_t s) {
  with_shape<T, 3>(a.tile, [&](auto G) {
    using GG = decltype(G);
    launch_k(k_strip_post<T, TO, GG>, strip_grid<GG>(a.g), GG::NT, strip_smem<GG, T>(true), s, a, x_in, xc, b,
             x_out, mx_out, out, oscale);
  });
}
template <typename T, typename TZ>
void launch_tile_amass(const TileMass<T>& a, const double* v, TZ* z1, T* t_out, cudaStream_t s) {
  using Mass = typename StripCfg<T>::Mass;
  launch_k(k_strip_amass<T, TZ, Mass, 0, QSPLIT, true, false>, strip_grid<Mass>(a.g), Mass::NT,
           strip_smem<Mass, T>(false), s, a, v, z1, t_out);
  launch_k(k_strip_amass<T, TZ, Mass, QSPLIT, QTILE - 1, false, true>, strip_grid<Mass>(a.g), Mass::NT,
           strip_smem<Mass, T>(false), s, a, v, z1, t_out);
}

template <typename T>
void launch_tile_pre_b(const StripPreItem<T>* items, int count, cudaStream_t s) {
  Batch<StripPreItem<T>> B;
  for (int i = 0; i < count; ++i) B.a[i] = items[i];
  const TileSmooth<T>& a = items[0].a;
  with_shape<T, 4>(a.tile, [&](auto G) {
    using GG = decltype(G);
    dim3 gr = strip_grid<GG>(a.g);
    gr.z = count;
    launch_k(k_strip_pre_b<T, GG>, gr, GG::NT, strip_smem<GG, T>(false), s, B);
  });
}
template <typename T, typename TO>
void launch_tile_post_b(const StripPostItem<T, TO>* items, int count, cudaStream_t s) {
  Batch<StripPostItem<T, TO>> B;
  for (int i = 0; i < count; ++i) B.a[i] = items[i];
  const TileSmooth<T>& a = items[0].a;
  with_shape<T, 3>(a.tile, [&](auto G) {
    using GG = decltype(G);
    dim3 gr = strip_grid<GG>(a.g);
    gr.z = count;
    launch_k(k_strip_post_b<T, TO, GG>, gr, GG::NT, strip_smem<GG, T>(true), s, B);
  });
}
template <typename T, typename TZ>
void launch_tile_amass_b(const AmassItem<T, TZ>* items, int count, cudaStream_t s) {
  using Mass = typename StripCfg<T>::Mass;
  Batch<AmassItem<T, TZ>> B;
  for (int i = 0; i < count; ++i) B.a[i] = items[i];
  dim3 gr = strip_grid<Mass>(items[0].a.g);
  gr.z = count;
  launch_k(k_strip_amass_b<T, TZ, Mass, 0, QSPLIT, true, false>, gr, Mass::NT, strip_smem<Mass, T>(false), s, B);
  launch_k(k_strip_amass_b<T, TZ, Mass, QSPLIT, QTILE - 1, false, true>, gr, Mass::NT, strip_smem<Mass, T>(false), s,
           B);
}

template <typename T>
cudaError_t prepare_tiles(int q) {
  (void)q;
  using MA = typename StripCfg<T>::Mass;
  const cudaFuncAttribute attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaSuccess;
  auto set = [&](auto kernel, size_t bytes) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kernel, attr, (int)bytes);
  };
  for (int sh = 0; sh < STRIP_SHAPES; ++sh) {
    with_shape<T, 4>(sh, [&](auto G) {
      using GG = decltype(G);
      set(k_strip_pre<T, GG>, strip_smem<GG, T>(false));
      set(k_strip_pre_b<T, GG>, strip_smem<GG, T>(false));
    });
    with_shape<T, 3>(sh, [&](auto G) {
      using GG = decltype(G);
      const size_t m = strip_smem<GG, T>(true);
      set(k_strip_post<T, float, GG>, m);
      set(k_strip_post<T, double, GG>, m);
      set(k_strip_post_b<T, T, GG>, m);
      if constexpr (std::is_same<T, float>::value) {
        set(k_strip_post<T, __half, GG>, m);
        set(k_strip_post_b<T, __half, GG>, m);
      }
    });
  }
  const size_t ms = strip_smem<MA, T>(false);
  set(k_strip_amass<T, float, MA, 0, QSPLIT, true, false>, ms);
  set(k_strip_amass<T, float, MA, QSPLIT, QTILE - 1, false, true>, ms);
  set(k_strip_amass<T, double, MA, 0, QSPLIT, true, false>, ms);
  set(k_strip_amass<T, double, MA, QSPLIT, QTILE - 1, false, true>, ms);
  if constexpr (std::is_same<T, float>::value) {
    set(k_strip_amass<T, __half, MA, 0, QSPLIT, true, false>, ms);
    set(k_strip_amass<T, __half, MA, QSPLIT, QTILE - 1, false, true>, ms);
    set(k_strip_amass_b<T, float, MA, 0, QSPLIT, true, false>, ms);
    set(k_strip_amass_b<T, float, MA, QSPLIT, QTILE - 1, false, true>, ms);
    set(k_strip_amass_b<T, __half, MA, 0, QSPLIT, true, false>, ms);
    set(k_strip_amass_b<T, __half, MA, QSPLIT, QTILE - 1, false, true>, ms);
  } else {
    set(k_strip_amass_b<T, double, MA, 0, QSPLIT, true, false>, ms);
    set(k_strip_amass_b<T, double, MA, QSPLIT, QTILE - 1, false, true>, ms);
  }
  return e;
}

// blocks of the pre-smoothing kernel on a level with the large (64) or small (32) window
template <typename T>
long long strip_blocks(const Geom& g, int tile) {
  long long n = 0;
  with_shape<T, 4>(tile, [&](auto G) {
    const dim3 d = strip_grid<decltype(G)>(g);
    n = (long long)d.x * d.y;
  });
  return n;
}

#define OK_TILE_INST(T)                                                                                       \
  template void launch_tile_pre<T>(const TileSmooth<T>&, const T*, const T*, T*, T*, cudaStream_t);           \
  template void launch_tile_post<T, T>(const TileSmooth<T>&, const T*, const T*, const T*, T*, T*, T*, T,     \
                                       cudaStream_t);                                                         \
  template void launch_tile_amass<T, T>(const TileMass<T>&, const double*, T*, T*, cudaStream_t);             \
  template cudaError_t prepare_tiles<T>(int);                                                                 \
  template long long strip_blocks<T>(const Geom&, int);                                                       \
  template int prepare_low_vcycle<T>(long long);                                                              \
  template void launch_low_vcycle<T>(const LowArgs<T>&, int, cudaStream_t);
OK_TILE_INST(float)
OK_TILE_INST(double)
template void launch_tile_post<float, double>(const TileSmooth<float>&, const float*, const float*, const float*,
                                              float*, float*, double*, float, cudaStream_t);
template void launch_tile_post<double, float>(const TileSmooth<double>&, const double*, const double*,
                                              const double*, double*, double*, float*, double, cudaStream_t);
template void launch_tile_amass<float, double>(const TileMass<float>&, const double*, double*, float*, cudaStream_t);
template void launch_tile_amass<double, float>(const TileMass<double>&, const double*, float*, double*,
                                               cudaStream_t);
template void launch_tile_post<float, __half>(const TileSmooth<float>&, const float*, const float*, const float*,
                                              float*, float*, __half*, float, cudaStream_t);
template void launch_tile_amass<float, __half>(const TileMass<float>&, const double*, __half*, float*,
                                               cudaStream_t);
template void launch_tile_pre_b<float>(const StripPreItem<float>*, int, cudaStream_t);
template void launch_tile_pre_b<double>(const StripPreItem<double>*, int, cudaStream_t);
template void launch_tile_post_b<float, float>(const StripPostItem<float, float>*, int, cudaStream_t);
template void launch_tile_post_b<float, __half>(const StripPostItem<float, __half>*, int, cudaStream_t);
template void launch_tile_post_b<double, double>(const StripPostItem<double, double>*, int, cudaStream_t);
template void launch_tile_amass_b<float, float>(const AmassItem<float, float>*, int, cudaStream_t);
template void launch_tile_amass_b<float, __half>(const AmassItem<float, __half>*, int, cudaStream_t);
template void launch_tile_amass_b<double, double>(const AmassItem<double, double>*, int, cudaStream_t);

}  // namespace okg
