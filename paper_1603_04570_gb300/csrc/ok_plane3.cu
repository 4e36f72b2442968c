// ok_plane3.cu -- 3D stencil steps by z-marching thread blocks.
//
// A thread block owns a PX x PY tile of (x, y) columns, one thread per column,
// and walks a chunk of pz consecutive z-planes (four compiled tile shapes,
// chosen per level by timing at setup; pz is chosen at launch so that the
// blocks fill whole waves of the SMs, see plane_chunk).  The vector the stencil reads is staged
// plane by plane into a ring of four shared-memory planes of (PY + 2) x
// (PX + 2) values (the tile and a one-vertex ring around it, zero outside the
// domain, which is the value load_nb gives an absent neighbour).  The 15
// couplings of the Kuhn P1 stencil of vertex (x, y, z) then come from planes
// z - 1, z, z + 1 of the ring:
//   plane z:     self, +-x, +-y, +-(x+y)
//   plane z + 1: +z, +(x+z), +(y+z), +(x+y+z)
//   plane z - 1: -z, -(x+z), -(y+z), -(x+y+z)
// so every value of the stencil vector is read from global memory once per
// block (plus the one-vertex ring), coalesced along x.  Plane z + 2 is
// fetched into registers while plane z is computed; with four ring slots one
// barrier per plane orders the writes of plane z + 1 after every read of the
// plane it replaces (z - 3).
//
// Each vertex update is the arithmetic of the per-vertex bodies of
// ok_stencil.cuh (cheb_step_at, resid_init_at, cheb_last_at) and of
// k_op_apply, with the same operands in the same order, so the results are
// bitwise those of the one-thread-per-vertex kernels.
#include "ok_internal.cuh"
#include "ok_kernels.h"
#include "ok_stencil.cuh"

#include <map>
#include <mutex>
#include <tuple>

namespace okg {

// Block shapes (PX x PY columns; PZ is the plane count the shape was first
// tuned with, kept as its name); the autotuner of the multigrid setup picks
// one per level by timing (all give the same bits).
template <int PX_, int PY_, int PZ_> struct PShape {
  static constexpr int PX = PX_, PY = PY_, PZ = PZ_;
  static constexpr int PW = PX + 2, PH = PY + 2;            // padded plane
  static constexpr int PNT = PX * PY;                       // threads
  static constexpr int PSLOT = (PW * PH + PNT - 1) / PNT;   // padded-plane elements staged per thread
};
using PShape0 = PShape<32, 8, 16>;
using PShape1 = PShape<32, 4, 32>;
using PShape2 = PShape<64, 4, 16>;
using PShape3 = PShape<32, 8, 32>;
constexpr int NTAB3 = Topo<3>::NCLASS * Topo<3>::NOFF;


// the update of one vertex given its 15 stencil values (INT: interior class,
// weights in registers)
template <typename T, typename TS, typename TO, int MODE, bool INT>
__device__ __forceinline__ void plane_update(const PlaneArgs<T, TS, TO>& a, const RegW<3, T>& rw, const T* sW,
                                             const T* sD, int cls, const T (&xs)[Topo<3>::NOFF], long long gi, T xv,
                                             T rv, T bv) {
  using Tp = Topo<3>;
  if constexpr (MODE == PM_OP) {
    T acc;
    if (a.axis_only) {
      if constexpr (INT) {
        acc = rw.w[0] * xs[0];
#pragma unroll
        for (int o = 1; o < Tp::NAX; ++o) acc = fma(rw.w[o], xs[o], acc);
      } else {
        acc = dot_w<3, Tp::NAX>(sW, cls, xs);
      }
    } else {
      if constexpr (INT) acc = dot_r<3, T>(rw, xs);
      else acc = dot_w<3, Tp::NOFF>(sW, cls, xs);
    }
    acc *= a.alpha;
    if (a.y0) acc = fma(a.beta, (T)a.y0[gi], acc);
    a.out[gi] = (TO)acc;
  } else {
    T dot;
    if constexpr (INT) dot = dot_r<3, T>(rw, xs);
    else dot = dot_w<3, Tp::NOFF>(sW, cls, xs);
    const T dv = INT ? rw.dinv : (MODE == PM_LAST ? (T)0 : sD[cls]);
    if constexpr (MODE == PM_RESID) {
      T rr = bv - dot;
      a.r[gi] = rr;
      a.d[gi] = dv * rr * a.inv_th;
    } else if constexpr (MODE == PM_STEP) {
      a.x[gi] = (a.first ? (T)0 : xv) + xs[0];
      T rr = rv - dot;
      a.r[gi] = rr;
      a.d[gi] = fma(a.c1, xs[0], a.c2 * (dv * rr));
    } else {                                        // PM_LAST (with the residual)
      T xx = (a.first ? (T)0 : xv) + xs[0];
      a.r[gi] = rv - dot;
      a.x[gi] = xx;
      if (a.out) a.out[gi] = (TO)(xx * a.oscale);
    }
  }
}

template <typename T, typename TS, typename TO, int MODE, class C>
__device__ __forceinline__ void plane3_body(const PlaneArgs<T, TS, TO>& a, int zchunk, int pz) {
  using Tp = Topo<3>;
  constexpr int PX = C::PX, PY = C::PY, PW = C::PW, PH = C::PH, PNT = C::PNT, PSLOT = C::PSLOT;
  __shared__ T sW[NTAB3];
  __shared__ T sD[Tp::NCLASS];
  __shared__ T ring[4][PH][PW];
  pdl_launch_dependents();
  for (int i = threadIdx.x; i < NTAB3; i += PNT) sW[i] = a.W[i];
  if (MODE != PM_OP && MODE != PM_LAST)
    for (int i = threadIdx.x; i < Tp::NCLASS; i += PNT) sD[i] = a.dinv[i];
  const Geom g = a.g;
  const int n = g.n;
  const int tx = threadIdx.x % PX, ty = threadIdx.x / PX;
  const int gx = blockIdx.x * PX + tx, gy = blockIdx.y * PY + ty;
  const int z0 = zchunk * pz;
  const int z1 = min(z0 + pz, n + 1);
  // padded-plane elements this thread stages: (ey, ex) -> global (x0 + ex - 1, y0 + ey - 1)
  long long eoff[PSLOT];
  bool ein[PSLOT];
  int ey[PSLOT], ex[PSLOT];
#pragma unroll
  for (int k = 0; k < PSLOT; ++k) {
    const int e = threadIdx.x + k * PNT;
    ey[k] = e / PW;
    ex[k] = e % PW;
    const int xx = blockIdx.x * PX + ex[k] - 1, yy = blockIdx.y * PY + ey[k] - 1;
    ein[k] = e < PW * PH && xx >= 0 && xx <= n && yy >= 0 && yy <= n;
    eoff[k] = ein[k] ? (long long)xx + g.sy * yy : 0;
  }
  const bool mine = gx <= n && gy <= n;
  const long long col = mine ? (long long)gx + g.sy * gy : 0;
  const int cx = axis_class(gx, n), cy = axis_class(gy, n);
  const int bx0 = blockIdx.x * PX, by0 = blockIdx.y * PY;
  const bool tile_int = bx0 >= 1 && bx0 + PX - 1 <= n - 1 && by0 >= 1 && by0 + PY - 1 <= n - 1;
  __syncthreads();                                  // tables staged
  RegW<3, T> rw = reg_weights<3, T>(sW, sD, 13);    // interior class (sD unused by OP / LAST)
  pdl_wait();                                       // the tables are fixed at setup; the rest is not
  // software pipeline: the stencil vector is fetched three planes ahead (two
  // register sets), the pointwise operands one plane ahead, so that several
  // planes' loads are in flight per warp
  T q0[PSLOT], q1[PSLOT];
  auto fetch = [&](int z, T (&q)[PSLOT]) {
#pragma unroll
    for (int k = 0; k < PSLOT; ++k)
      q[k] = (ein[k] && z >= 0 && z <= n) ? (T)a.s[eoff[k] + g.sz * z] : (T)0;
  };
  auto stage = [&](int z, const T (&q)[PSLOT]) {
#pragma unroll
    for (int k = 0; k < PSLOT; ++k)
      if (threadIdx.x + k * PNT < PW * PH) ring[z & 3][ey[k]][ex[k]] = q[k];
  };
  struct Pw { T x, r, b; };
  auto pointwise = [&](int z) {
    Pw p{(T)0, (T)0, (T)0};
    if (mine && z < z1) {
      const long long gi = col + g.sz * z;
      if (MODE == PM_RESID) p.b = a.b[gi];
      if ((MODE == PM_STEP || MODE == PM_LAST) && !a.first) p.x = a.x[gi];
      if (MODE == PM_STEP || MODE == PM_LAST) p.r = a.r[gi];
    }
    return p;
  };
  fetch(z0 - 1, q0);
  stage(z0 - 1, q0);
  fetch(z0, q0);
  stage(z0, q0);
  fetch(z0 + 1, q0);
  fetch(z0 + 2, q1);
  Pw cur = pointwise(z0);
  const int lx = tx + 1, ly = ty + 1;
  for (int z = z0; z < z1; ++z) {
    stage(z + 1, q0);
#pragma unroll
    for (int k = 0; k < PSLOT; ++k) q0[k] = q1[k];
    if (z + 2 < z1) fetch(z + 3, q1);
    const Pw nxt = pointwise(z + 1);
    const long long gi = col + g.sz * z;
    const T xv = cur.x, rv = cur.r, bv = cur.b;
    cur = nxt;
    __syncthreads();
    if (!mine) continue;
    const T(*pm)[PW] = ring[(z + 3) & 3];
    const T(*p0)[PW] = ring[z & 3];
    const T(*pp)[PW] = ring[(z + 1) & 3];
    T xs[Tp::NOFF];
    xs[0] = p0[ly][lx];
    xs[1] = p0[ly][lx + 1];
    xs[2] = p0[ly][lx - 1];
    xs[3] = p0[ly + 1][lx];
    xs[4] = p0[ly - 1][lx];
    xs[5] = pp[ly][lx];
    xs[6] = pm[ly][lx];
    xs[7] = p0[ly + 1][lx + 1];
    xs[8] = p0[ly - 1][lx - 1];
    xs[9] = pp[ly][lx + 1];
    xs[10] = pm[ly][lx - 1];
    xs[11] = pp[ly + 1][lx];
    xs[12] = pm[ly - 1][lx];
    xs[13] = pp[ly + 1][lx + 1];
    xs[14] = pm[ly - 1][lx - 1];
    // a plane of a tile whose columns are all interior holds only interior
    // vertices: the branch is uniform over the block, and each side computes
    // one dot product (weights in registers, or the class table)
    if (tile_int && z >= 1 && z <= n - 1) plane_update<T, TS, TO, MODE, true>(a, rw, sW, sD, 13, xs, gi, xv, rv, bv);
    else plane_update<T, TS, TO, MODE, false>(a, rw, sW, sD, cx + 3 * cy + 9 * axis_class(z, n), xs, gi, xv, rv, bv);
  }
}
template <typename T, typename TS, typename TO, int MODE, class C>
__global__ void __launch_bounds__(C::PNT) k_plane3(PlaneArgs<T, TS, TO> a, int pz) {
  plane3_body<T, TS, TO, MODE, C>(a, blockIdx.z, pz);
}
// batched: blockIdx.z = problem * (z-chunks) + chunk
template <typename T, typename TS, typename TO, int MODE, class C>
__global__ void __launch_bounds__(C::PNT) k_plane3_b(Batch<PlaneArgs<T, TS, TO>> B, int nzc, int pz) {
  plane3_body<T, TS, TO, MODE, C>(B.a[blockIdx.z / nzc], blockIdx.z % nzc, pz);
}

// Planes per block.  A launch of T column tiles split into c z-chunks runs in
// ceil(T c / R) waves of R = (resident blocks per SM) x (SMs) blocks, each
// block walking ceil(n1 / c) planes after staging two; c is chosen to
// minimise waves x (planes + 2).  (At 129^3 with 32 x 8 tiles and four
// resident blocks per SM this gives 7 chunks of 19 planes, one wave, where
// fixed 16-plane chunks need 765 blocks: 1.26 waves.)  Every plane is
// computed once whatever c is, so the results do not depend on it.
static int plane_chunk(const void* kern, int pnt, int n1, long long tiles) {
  int dev = 0;
  cudaGetDevice(&dev);
  static std::mutex mu;
  static std::map<std::tuple<const void*, int, long long, int>, int> cache;
  std::lock_guard<std::mutex> lk(mu);
  const auto key = std::make_tuple(kern, n1, tiles, dev);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int nsm = 0, per_sm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, pnt, 0) != cudaSuccess) {
    cudaGetLastError();
    per_sm = 1;
  }
  const long long R = (long long)(nsm > 0 ? nsm : 1) * (per_sm > 0 ? per_sm : 1);
  int best_pz = n1;
  long long best = -1;
  for (int c = 1; c <= n1; ++c) {
    const int pz = (n1 + c - 1) / c;
    const int chunks = (n1 + pz - 1) / pz;
    if (chunks != c) continue;                       // same pz as a smaller c
    const long long cost = ((tiles * chunks + R - 1) / R) * (pz + 2);
    if (best < 0 || cost < best) {
      best = cost;
      best_pz = pz;
    }
  }
  // Where 32-plane chunks already make two waves or more (the large, HBM-bound
  // levels), they are kept: measured faster there than the model's longer
  // chunks (257^3: 114 against 127 us per Chebyshev step; 513^3: 828 against
  // 842 us), the model's waves x planes not seeing what longer marches cost.
  const int c32 = (n1 + 31) / 32;
  if (best_pz > 32 && tiles * c32 >= 2 * R) best_pz = (n1 + c32 - 1) / c32;
  cache[key] = best_pz;
  return best_pz;
}

template <class C>
static inline long long plane_tiles(const Geom& g) {
  return (long long)((g.n1 + C::PX - 1) / C::PX) * ((g.n1 + C::PY - 1) / C::PY);
}

template <typename T, typename TS, typename TO, int MODE, class C>
static void launch_plane1(const PlaneArgs<T, TS, TO>& a, cudaStream_t s) {
  auto kern = k_plane3<T, TS, TO, MODE, C>;
  const int pz = plane_chunk((const void*)kern, C::PNT, a.g.n1, plane_tiles<C>(a.g));
  const dim3 gr((a.g.n1 + C::PX - 1) / C::PX, (a.g.n1 + C::PY - 1) / C::PY, (a.g.n1 + pz - 1) / pz);
  launch_k(kern, gr, C::PNT, 0, s, a, pz);
}

template <typename T, typename TS, typename TO, int MODE>
static void launch_plane(const PlaneArgs<T, TS, TO>& a, int shape, cudaStream_t s) {
  switch (shape) {
    case 1: launch_plane1<T, TS, TO, MODE, PShape1>(a, s); break;
    case 2: launch_plane1<T, TS, TO, MODE, PShape2>(a, s); break;
    case 3: launch_plane1<T, TS, TO, MODE, PShape3>(a, s); break;
    default: launch_plane1<T, TS, TO, MODE, PShape0>(a, s);
  }
}

template <typename T, typename TS, typename TO, int MODE, class C>
static void launch_plane_b1(const Batch<PlaneArgs<T, TS, TO>>& B, const Geom& g, int count, cudaStream_t s) {
  auto kern = k_plane3_b<T, TS, TO, MODE, C>;
  const int pz = plane_chunk((const void*)kern, C::PNT, g.n1, plane_tiles<C>(g) * count);
  const int nzc = (g.n1 + pz - 1) / pz;
  const dim3 gr((g.n1 + C::PX - 1) / C::PX, (g.n1 + C::PY - 1) / C::PY, nzc * count);
  launch_k(kern, gr, C::PNT, 0, s, B, nzc, pz);
}
template <typename T, typename TS, typename TO>
void launch_plane3_b(int mode, const PlaneArgs<T, TS, TO>* items, int count, int shape, cudaStream_t s) {
  Batch<PlaneArgs<T, TS, TO>> B;
  for (int i = 0; i < count; ++i) B.a[i] = items[i];
  const Geom& g = items[0].g;
  auto go = [&](auto M) {
    constexpr int MODE = decltype(M)::value;
    switch (shape) {
      case 1: launch_plane_b1<T, TS, TO, MODE, PShape1>(B, g, count, s); break;
      case 2: launch_plane_b1<T, TS, TO, MODE, PShape2>(B, g, count, s); break;
      case 3: launch_plane_b1<T, TS, TO, MODE, PShape3>(B, g, count, s); break;
      default: launch_plane_b1<T, TS, TO, MODE, PShape0>(B, g, count, s);
    }
  };
  switch (mode) {
    case PM_RESID: go(std::integral_constant<int, PM_RESID>{}); break;
    case PM_STEP: go(std::integral_constant<int, PM_STEP>{}); break;
    case PM_LAST: go(std::integral_constant<int, PM_LAST>{}); break;
    default: go(std::integral_constant<int, PM_OP>{});
  }
}

template <typename T>
void launch_resid_init3(const Geom& g, const T* W, const T* dinv, const T* b, const T* x, T* r, T* d, T inv_th,
                        cudaStream_t s, int shape) {
  PlaneArgs<T, T, T> a = {};
  a.g = g;
  a.W = W;
  a.dinv = dinv;
  a.s = x;
  a.r = r;
  a.d = d;
  a.b = b;
  a.inv_th = inv_th;
  launch_plane<T, T, T, PM_RESID>(a, shape, s);
}

template <typename T>
void launch_cheb_step3(const Geom& g, const T* W, const T* dinv, T* x, T* r, const T* d_in, T* d_out, T c1, T c2,
                       bool first, cudaStream_t s, int shape) {
  PlaneArgs<T, T, T> a = {};
  a.g = g;
  a.W = W;
  a.dinv = dinv;
  a.s = d_in;
  a.x = x;
  a.r = r;
  a.d = d_out;
  a.c1 = c1;
  a.c2 = c2;
  a.first = first ? 1 : 0;
  launch_plane<T, T, T, PM_STEP>(a, shape, s);
}

template <typename T, typename TO>
void launch_cheb_last3(const Geom& g, const T* W, T* x, T* r, const T* d_in, bool first, TO* out, T oscale,
                       cudaStream_t s, int shape) {
  PlaneArgs<T, T, TO> a = {};
  a.g = g;
  a.W = W;
  a.s = d_in;
  a.x = x;
  a.r = r;
  a.out = out;
  a.oscale = oscale;
  a.first = first ? 1 : 0;
  launch_plane<T, T, TO, PM_LAST>(a, shape, s);
}

template <typename T, typename TX, typename TY>
void launch_op_apply3(const Geom& g, const T* W, bool axis_only, const TX* x, TY* y, T alpha, const TY* y0, T beta,
                      cudaStream_t s, int shape) {
  PlaneArgs<T, TX, TY> a = {};
  a.g = g;
  a.W = W;
  a.s = x;
  a.out = y;
  a.y0 = y0;
  a.alpha = alpha;
  a.beta = beta;
  a.axis_only = axis_only ? 1 : 0;
  launch_plane<T, TX, TY, PM_OP>(a, shape, s);
}

#define OK_PLANE_INST(T)                                                                                      \
  template void launch_resid_init3<T>(const Geom&, const T*, const T*, const T*, const T*, T*, T*, T,         \
                                      cudaStream_t, int);                                                     \
  template void launch_cheb_step3<T>(const Geom&, const T*, const T*, T*, T*, const T*, T*, T, T, bool,       \
                                     cudaStream_t, int);                                                      \
  template void launch_cheb_last3<T, T>(const Geom&, const T*, T*, T*, const T*, bool, T*, T, cudaStream_t,   \
                                        int);                                                                 \
  template void launch_op_apply3<T, T, T>(const Geom&, const T*, bool, const T*, T*, T, const T*, T,          \
                                          cudaStream_t, int);
OK_PLANE_INST(float)
OK_PLANE_INST(double)
template void launch_plane3_b<float, float, float>(int, const PlaneArgs<float, float, float>*, int, int,
                                                   cudaStream_t);
template void launch_plane3_b<double, double, double>(int, const PlaneArgs<double, double, double>*, int, int,
                                                      cudaStream_t);
template void launch_cheb_last3<float, double>(const Geom&, const float*, float*, float*, const float*, bool,
                                               double*, float, cudaStream_t, int);
template void launch_cheb_last3<float, __half>(const Geom&, const float*, float*, float*, const float*, bool,
                                               __half*, float, cudaStream_t, int);
template void launch_cheb_last3<double, float>(const Geom&, const double*, double*, double*, const double*, bool,
                                               float*, double, cudaStream_t, int);

}  // namespace okg
