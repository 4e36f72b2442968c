// ok_stencil.cuh -- per-vertex bodies of the Chebyshev, transfer and coarse
// steps, shared by every kernel that performs them (one kernel per step, the
// fused coarse V-cycle, the shared-memory tile kernels), so that all paths
// take the same arithmetic in the same order and round identically.  Every
// product that feeds a sum is an explicit fma.
#pragma once

#include "ok_internal.cuh"

namespace okg {

template <int D, typename T, typename TB>
__device__ __forceinline__ void cheb_init_at(const Vtx<D>& v, const T* dinv, const TB* b, T bscale, T* r, T* d,
                                             T inv_th) {
  T rr = (T)b[v.idx] * bscale;
  r[v.idx] = rr;
  d[v.idx] = dinv[v.cls] * rr * inv_th;
}

template <int D, typename T>
__device__ __forceinline__ void resid_init_at(const Geom& g, const Vtx<D>& v, const T* W, const T* dinv,
                                              const T* b, const T* x, T* r, T* d, T inv_th) {
  T xs[Topo<D>::NOFF];
  load_nb<D>(x, g, v, xs);
  T rr = b[v.idx] - dot_w<D, Topo<D>::NOFF>(W, v.cls, xs);
  r[v.idx] = rr;
  d[v.idx] = dinv[v.cls] * rr * inv_th;
}

template <int D, typename T>
__device__ __forceinline__ void cheb_step_at(const Geom& g, const Vtx<D>& v, const T* W, const T* dinv, T* x,
                                             T* r, const T* din, T* dout, T c1, T c2, bool first) {
  T ds[Topo<D>::NOFF];
  load_nb<D>(din, g, v, ds);
  x[v.idx] = (first ? (T)0 : x[v.idx]) + ds[0];
  T rr = r[v.idx] - dot_w<D, Topo<D>::NOFF>(W, v.cls, ds);
  r[v.idx] = rr;
  dout[v.idx] = fma(c1, ds[0], c2 * (dinv[v.cls] * rr));
}

template <int D, typename T, typename TO>
__device__ __forceinline__ void cheb_last_at(const Geom& g, const Vtx<D>& v, const T* W, T* x, T* r,
                                             const T* din, bool first, TO* out, T oscale) {
  T xx;
  if (r) {
    T ds[Topo<D>::NOFF];
    load_nb<D>(din, g, v, ds);
    xx = (first ? (T)0 : x[v.idx]) + ds[0];
    r[v.idx] = r[v.idx] - dot_w<D, Topo<D>::NOFF>(W, v.cls, ds);
  } else {
    xx = (first ? (T)0 : x[v.idx]) + din[v.idx];
  }
  x[v.idx] = xx;
  if (out) out[v.idx] = (TO)(xx * oscale);
}

// v: coarse vertex (position p), gf: fine geometry
template <int D, typename T>
__device__ __forceinline__ void restrict_at(const Geom& gf, const Vtx<D>& v, const T* rf, T* bc) {
  long long fc = 2LL * v.p[0] + gf.sy * (2LL * v.p[1]) + gf.sz * (2LL * v.p[2]);
  T acc = (T)0;
  static_for<1, Topo<D>::NOFF>([&](auto O) {
    constexpr int o = decltype(O)::value;
    if (nb_valid<D, o>(v.c)) acc += rf[fc + nb_delta<D, o>(gf)];
  });
  bc[v.idx] = fma((T)0.5, acc, rf[fc]);
}

// v: fine vertex, gc: coarse geometry.  With dc, the coarse iterate is
// xc + dc, rounded as the last smoothing step (cheb_last_at without r) rounds
// it: the coarse level's last step is folded into this launch.
template <int D, typename T>
__device__ __forceinline__ void prolong_add_at(const Geom& gc, const Vtx<D>& v, T* xf, const T* xc,
                                               const T* dc = nullptr) {
  long long ci = 0, cj = 0;
  bool mid = false;
  const long long st[3] = {1, gc.sy, gc.sz};
#pragma unroll
  for (int a = 0; a < D; ++a) {
    ci += (long long)(v.p[a] >> 1) * st[a];
    cj += (long long)((v.p[a] >> 1) + (v.p[a] & 1)) * st[a];
    mid = mid || (v.p[a] & 1);
  }
  const T ai = dc ? xc[ci] + dc[ci] : xc[ci];
  if (mid) {
    const T aj = dc ? xc[cj] + dc[cj] : xc[cj];
    xf[v.idx] = fma((T)0.5, ai + aj, xf[v.idx]);
  } else {
    xf[v.idx] = xf[v.idx] + ai;
  }
}

// x[r] = sum_c A[r][c] b[c] for the rows of this warp, xor-reduced.  Lane l
// takes the 16-byte groups l, l + 32, ... (E = 16 / sizeof(T) columns each, in
// column order): the order of the many-block GEMV with vector loads.
template <typename T>
__device__ __forceinline__ void coarse_rows(long long nc, const T* A, const T* b, T* x, int warp, int nw) {
  constexpr int E = 16 / sizeof(T);
  const int lane = threadIdx.x & 31;
  for (long long r = warp; r < nc; r += nw) {
    T acc = (T)0;
    for (long long c4 = lane; c4 * E < nc; c4 += 32)
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const long long c = c4 * E + e;
        if (c < nc) acc = fma(A[r * nc + c], b[c], acc);
      }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) x[r] = acc;
  }
}

// ---------------------------------------------------------------------------
// Dense coarsest-level GEMV with 16-byte loads.  The inverse has a padded row
// stride ld (a multiple of 16 bytes, zeros beyond column nc); b is staged in
// shared memory, zero-padded to whole chunks of 32 * GEMV_NPL vectors.  Lane l
// takes the vectors l, l + 32, ... in order, so the sum is that of coarse_rows.
// ---------------------------------------------------------------------------
constexpr int GEMV_NPL = 9;          // 16-byte vectors per lane per chunk (a 1089-wide float row in one)
template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; static constexpr int E = 4; };
template <> struct Vec16<double> { using type = double2; static constexpr int E = 2; };
template <typename T>
__device__ __forceinline__ T vec_at(const typename Vec16<T>::type& v, int e);
template <> __device__ __forceinline__ float vec_at<float>(const float4& v, int e) {
  return e == 0 ? v.x : (e == 1 ? v.y : (e == 2 ? v.z : v.w));
}
template <> __device__ __forceinline__ double vec_at<double>(const double2& v, int e) { return e == 0 ? v.x : v.y; }
// 16-byte read-only loads kept in program order (volatile), so a lane's loads
// of one chunk are all in flight before the first multiply
__device__ __forceinline__ void ld16(const float4* p, float4& v) {
  asm volatile("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
}
__device__ __forceinline__ void ld16(const double2* p, double2& v) {
  asm volatile("ld.global.nc.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "l"(p));
}

// elements of the staged b (padded to whole chunks)
template <typename T>
__host__ __device__ inline long long gemv_staged(long long ld) {
  const long long E = Vec16<T>::E, chunk = 32LL * GEMV_NPL;
  const long long nvec = ld / E;
  return ((nvec + chunk - 1) / chunk) * chunk * E;
}

// sb[i] = b[i] (i < nc), 0 up to the padded length; CG: b may have been written
// by other blocks of the same launch (load through L2)
template <typename T, bool CG>
__device__ __forceinline__ void gemv_stage_b(long long nc, long long ld, const T* b, T* sb) {
  const long long nb = gemv_staged<T>(ld);
  for (long long i = threadIdx.x; i < nb; i += blockDim.x) sb[i] = i < nc ? (CG ? __ldcg(b + i) : b[i]) : (T)0;
}

// 16-byte vectors [base, base + 32 GEMV_NPL) of row Ar for this lane (zero beyond nvec)
template <typename T>
__device__ __forceinline__ void gemv_load(const typename Vec16<T>::type* Ar, long long nvec, long long base,
                                          typename Vec16<T>::type (&a)[GEMV_NPL]) {
  using V = typename Vec16<T>::type;
  const int lane = threadIdx.x & 31;
  if (base + 32LL * GEMV_NPL <= nvec) {               // full chunk: all loads issued first
#pragma unroll
    for (int k = 0; k < GEMV_NPL; ++k) ld16(Ar + base + lane + 32 * k, a[k]);
  } else {                                            // ragged last chunk
#pragma unroll
    for (int k = 0; k < GEMV_NPL; ++k) {
      const long long c = base + lane + 32 * k;
      a[k] = V{};
      if (c < nvec) ld16(Ar + c, a[k]);
    }
  }
}
template <typename T>
__device__ __forceinline__ void gemv_mac(const typename Vec16<T>::type (&a)[GEMV_NPL], const T* sb, long long base,
                                         T& acc) {
  using V = typename Vec16<T>::type;
  constexpr int E = Vec16<T>::E;
  const int lane = threadIdx.x & 31;
  const V* sv = reinterpret_cast<const V*>(sb);
#pragma unroll
  for (int k = 0; k < GEMV_NPL; ++k) {
    const V bv = sv[base + lane + 32 * k];
#pragma unroll
    for (int e = 0; e < E; ++e) acc = fma(vec_at<T>(a[k], e), vec_at<T>(bv, e), acc);
  }
}
// the chunks after the first (a0: the first, already loaded), then the warp sum
template <typename T>
__device__ __forceinline__ T gemv_finish(long long ld, const T* __restrict__ A, const T* sb, long long r,
                                         const typename Vec16<T>::type (&a0)[GEMV_NPL]) {
  using V = typename Vec16<T>::type;
  const long long nvec = ld / Vec16<T>::E;
  const V* Ar = reinterpret_cast<const V*>(A + r * ld);
  T acc = (T)0;
  gemv_mac<T>(a0, sb, 0, acc);
  for (long long base = 32LL * GEMV_NPL; base < nvec; base += 32LL * GEMV_NPL) {
    V a[GEMV_NPL];
    gemv_load<T>(Ar, nvec, base, a);
    gemv_mac<T>(a, sb, base, acc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  return acc;
}
// row r of A times the staged b, by one warp (result in every lane)
template <typename T>
__device__ __forceinline__ T gemv_row(long long ld, const T* __restrict__ A, const T* sb, long long r) {
  typename Vec16<T>::type a0[GEMV_NPL];
  gemv_load<T>(reinterpret_cast<const typename Vec16<T>::type*>(A + r * ld), ld / Vec16<T>::E, 0, a0);
  return gemv_finish<T>(ld, A, sb, r, a0);
}

// ---------------------------------------------------------------------------
// The same bodies with one class's weights held in registers (vertices all of
// that class, e.g. the interior of a tile): identical arithmetic and order.
// ---------------------------------------------------------------------------
template <int D, typename T> struct RegW {
  T w[Topo<D>::NOFF];
  T dinv;
};

template <int D, typename T>
__device__ __forceinline__ RegW<D, T> reg_weights(const T* W, const T* dinv, int cls) {
  RegW<D, T> r;
#pragma unroll
  for (int o = 0; o < Topo<D>::NOFF; ++o) r.w[o] = W[cls * Topo<D>::NOFF + o];
  r.dinv = dinv[cls];
  return r;
}

template <int D, typename T>
__device__ __forceinline__ T dot_r(const RegW<D, T>& rw, const T (&xs)[Topo<D>::NOFF]) {
  T acc = rw.w[0] * xs[0];
#pragma unroll
  for (int o = 1; o < Topo<D>::NOFF; ++o) acc = fma(rw.w[o], xs[o], acc);
  return acc;
}

template <int D, typename T>
__device__ __forceinline__ void cheb_init_r(const Vtx<D>& v, const RegW<D, T>& rw, const T* b, T* r, T* d, T inv_th) {
  T rr = b[v.idx] * (T)1;
  r[v.idx] = rr;
  d[v.idx] = rw.dinv * rr * inv_th;
}

template <int D, typename T>
__device__ __forceinline__ void resid_init_r(const Geom& g, const Vtx<D>& v, const RegW<D, T>& rw, const T* b,
                                             const T* x, T* r, T* d, T inv_th) {
  T xs[Topo<D>::NOFF];
  load_nb<D>(x, g, v, xs);
  T rr = b[v.idx] - dot_r<D, T>(rw, xs);
  r[v.idx] = rr;
  d[v.idx] = rw.dinv * rr * inv_th;
}

template <int D, typename T>
__device__ __forceinline__ void cheb_step_r(const Geom& g, const Vtx<D>& v, const RegW<D, T>& rw, T* x, T* r,
                                            const T* din, T* dout, T c1, T c2, bool first) {
  T ds[Topo<D>::NOFF];
  load_nb<D>(din, g, v, ds);
  x[v.idx] = (first ? (T)0 : x[v.idx]) + ds[0];
  T rr = r[v.idx] - dot_r<D, T>(rw, ds);
  r[v.idx] = rr;
  dout[v.idx] = fma(c1, ds[0], c2 * (rw.dinv * rr));
}

template <int D, typename T>
__device__ __forceinline__ void cheb_last_r(const Geom& g, const Vtx<D>& v, const RegW<D, T>& rw, T* x, T* r,
                                            const T* din, bool first) {
  T xx;
  if (r) {
    T ds[Topo<D>::NOFF];
    load_nb<D>(din, g, v, ds);
    xx = (first ? (T)0 : x[v.idx]) + ds[0];
    r[v.idx] = r[v.idx] - dot_r<D, T>(rw, ds);
  } else {
    xx = (first ? (T)0 : x[v.idx]) + din[v.idx];
  }
  x[v.idx] = xx;
}

// vertex data from a linear index (block-stride loops)
template <int D, typename T>
__device__ __forceinline__ void vertex_of_index(const Geom& g, long long idx, Vtx<D>& v) {
  const long long n1 = g.n1;
  v.idx = idx;
  v.p[0] = (int)(idx % n1);
  const long long rest = idx / n1;
  v.p[1] = (int)(rest % n1);
  v.p[2] = D == 3 ? (int)(rest / n1) : 0;
  v.c[0] = axis_class(v.p[0], g.n);
  v.c[1] = axis_class(v.p[1], g.n);
  v.c[2] = D == 3 ? axis_class(v.p[2], g.n) : 1;
  v.cls = v.c[0] + 3 * v.c[1] + (D == 3 ? 9 * v.c[2] : 0);
}


}  // namespace okg
