// ok_internal.cuh -- shared declarations of the GB300 Ohta--Kawasaki library.
//
// Mesh topology (uniform P1 simplices, Sec. 2 discretisation):
//   * vertex (i,j[,k]) -> index i + sy j + sz k, sy = n+1, sz = (n+1)^2;
//   * every simplex is a "path" simplex of a cell: vertices
//       0, e_pi(0), e_pi(0)+e_pi(1), ..., (1,..,1)
//     for a permutation pi of the axes (2 triangles per square split along the
//     (0,0)-(1,1) diagonal; the 6 Kuhn tetrahedra per cube);
//   * the P1 couplings of a vertex are the 2^(d+1)-1 offsets 0 and +-b,
//     b in {0,1}^d \ {0} (7 in 2D, 15 in 3D);
//   * K couples only the 2d axis neighbours (the path Laplacian of each
//     simplex has no entry between non-consecutive path vertices).
// Boundary handling: a vertex's "class" is (c_x, c_y[, c_z]) with
// c_a = 0 at coordinate 0, 2 at coordinate n, 1 inside; the assembled
// stencil weights of M and K depend only on the class, and are tabulated per
// grid level (9 classes in 2D, 27 in 3D).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <type_traits>
#include <utility>

#include <atomic>

namespace okg {

// Kernels launched by this process (host-side count; a launch inside stream
// capture is counted by the capturing code per graph replay instead).
extern std::atomic<long long> g_launch_count;
inline void count_launch() { g_launch_count.fetch_add(1, std::memory_order_relaxed); }

// Programmatic dependent launch: a kernel launched with launch_k may be
// scheduled while its predecessor on the stream is still running; every
// kernel therefore starts with pdl_entry(), which lets its own successor be
// scheduled and then waits (in hardware) until the predecessor has completed
// and its memory is visible.  Without the launch attribute both are no-ops.
extern thread_local bool g_pdl;
__device__ __forceinline__ void pdl_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_entry() {
  pdl_launch_dependents();
  pdl_wait();
}
// Kernels that read data fixed at setup (class tables, the coarse inverse)
// call pdl_launch_dependents() first, issue those reads, and only then
// pdl_wait() before touching what the previous kernel wrote.

template <typename... KP, typename... A>
inline void launch_k(void (*kernel)(KP...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A&&... args) {
  count_launch();
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = g_pdl ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

// ---------------------------------------------------------------------------
// compile-time topology
// ---------------------------------------------------------------------------
template <int D> struct Topo {
  static constexpr int NOFF = D == 2 ? 7 : 15;      // self + 2*NPOS
  static constexpr int NPOS = D == 2 ? 3 : 7;       // b in {0,1}^d \ {0}
  static constexpr int NAX = 2 * D + 1;             // self + axis offsets
  static constexpr int NPERM = D == 2 ? 2 : 6;      // simplices per cell
  static constexpr int NINC = NPERM * (D + 1);      // (simplex, vertex) incidences
  static constexpr int NCLASS = D == 2 ? 9 : 27;
  static constexpr int NSLOT = NPOS + 1;            // symmetric coefficient storage
  static constexpr int FACT = D == 2 ? 2 : 6;       // d!
};

// bit pattern of the p-th positive offset: 2D (1,0),(0,1),(1,1);
// 3D x, y, z, x+y, x+z, y+z, x+y+z.  The first d are the axes.
__host__ __device__ constexpr int pos_bits(int D, int p) {
  return D == 2 ? (p == 0 ? 1 : (p == 1 ? 2 : 3))
                : (p < 3 ? (1 << p) : (p == 3 ? 3 : (p == 4 ? 5 : (p == 5 ? 6 : 7))));
}
__host__ __device__ constexpr int pos_index(int D, int bits) {
  return D == 2 ? (bits == 1 ? 0 : (bits == 2 ? 1 : 2))
                : (bits == 1 ? 0 : bits == 2 ? 1 : bits == 4 ? 2 : bits == 3 ? 3
                   : bits == 5 ? 4 : bits == 6 ? 5 : 6);
}
// offset o: 0 = self, 2p+1 = +pos(p), 2p+2 = -pos(p); component along axis a
__host__ __device__ constexpr int off_comp(int D, int o, int a) {
  return o == 0 ? 0 : ((pos_bits(D, (o - 1) / 2) >> a) & 1) * ((o & 1) ? 1 : -1);
}
// axis moved at step i of the path of simplex s (permutations in lexicographic order)
__host__ __device__ constexpr int perm_axis(int D, int s, int i) {
  return D == 2 ? (s == 0 ? i : 1 - i)
                : (s == 0 ? i
                   : s == 1 ? (i == 0 ? 0 : (i == 1 ? 2 : 1))
                   : s == 2 ? (i == 0 ? 1 : (i == 1 ? 0 : 2))
                   : s == 3 ? (i == 0 ? 1 : (i == 1 ? 2 : 0))
                   : s == 4 ? (i == 0 ? 2 : (i == 1 ? 0 : 1))
                            : (2 - i));
}
// corner bits of path vertex k of simplex s
__host__ __device__ constexpr int path_bits(int D, int s, int k) {
  return k == 0 ? 0 : (path_bits(D, s, k - 1) | (1 << perm_axis(D, s, k - 1)));
}
// incidence i = (simplex s, position k of the centre vertex in it)
__host__ __device__ constexpr int inc_simplex(int D, int i) { return i / (D + 1); }
__host__ __device__ constexpr int inc_pos(int D, int i) { return i % (D + 1); }
// corner of the centre vertex inside the cell of incidence i; bit a set means
// the cell lies on the negative side along axis a (cell origin v - e_a)
__host__ __device__ constexpr int inc_corner(int D, int i) {
  return path_bits(D, inc_simplex(D, i), inc_pos(D, i));
}
// offset index (relative to the centre vertex) of vertex t of incidence i
__host__ __device__ constexpr int inc_off(int D, int i, int t) {
  return t == inc_pos(D, i) ? 0
       : (t > inc_pos(D, i)
            ? 2 * pos_index(D, path_bits(D, inc_simplex(D, i), t) & ~inc_corner(D, i)) + 1
            : 2 * pos_index(D, inc_corner(D, i) & ~path_bits(D, inc_simplex(D, i), t)) + 2);
}
// path Laplacian: unit-simplex stiffness d! K_T / h^(d-2)
__host__ __device__ constexpr int path_lap(int D, int a, int b) {
  return a == b ? ((a == 0 || a == D) ? 1 : 2) : ((a - b == 1 || b - a == 1) ? -1 : 0);
}

// compile-time loop
template <int B, int E, typename F>
__host__ __device__ __forceinline__ void static_for(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

// ---------------------------------------------------------------------------
// grid geometry passed to kernels
// ---------------------------------------------------------------------------
struct Geom {
  int n;           // cells per side
  int n1;          // n + 1
  long long nv;    // vertices
  long long sy;    // stride of y
  long long sz;    // stride of z (0 in 2D)
  unsigned rmul;   // ceil(2^32 / n1): t / n1 = umulhi(t, rmul) for 0 <= t < n1^2 while n1^3 < 2^32
};

inline Geom make_geom(int dim, int n) {
  Geom g;
  g.n = n;
  g.n1 = n + 1;
  g.sy = n + 1;
  g.sz = dim == 3 ? (long long)(n + 1) * (n + 1) : 0;
  g.nv = dim == 3 ? g.sz * (n + 1) : g.sy * (n + 1);
  g.rmul = (unsigned)((0x100000000ull + (unsigned long long)g.n1 - 1) / (unsigned long long)g.n1);
  return g;
}

__device__ __forceinline__ int axis_class(int i, int n) { return i == 0 ? 0 : (i == n ? 2 : 1); }

// Per-vertex position data: index, class per axis and the linear class.
template <int D> struct Vtx {
  long long idx;
  int p[3];      // grid coordinates (i, j, k)
  int c[3];
  int cls;
};

// thread -> vertex for the launch shape grid(ceil(n1^2 / bx), 1, D==3 ? n1 : 1)
// (kz: the z-plane; batched launches fold the problem index into blockIdx.z).
// The threads of a block take consecutive vertices of one (x, y) plane, rows
// back to back, so that no warp idles at the end of a row of 2^k + 1 vertices.
template <int D>
__device__ __forceinline__ bool vertex_of_thread_at(const Geom& g, int kz, Vtx<D>& v) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.n1 * g.n1) return false;
  // t / n1 by a multiply where that is exact (t n1 < n1^3 < 2^32: the
  // quotient's error t (rmul n1 - 2^32) / 2^32 n1 stays below 1 / n1)
  const int j = g.n1 <= 1625 ? (int)__umulhi((unsigned)t, g.rmul) : t / g.n1;
  const int i = t - j * g.n1;
  int k = D == 3 ? kz : 0;
  v.p[0] = i;
  v.p[1] = j;
  v.p[2] = k;
  v.idx = i + g.sy * j + g.sz * k;
  v.c[0] = axis_class(i, g.n);
  v.c[1] = axis_class(j, g.n);
  v.c[2] = D == 3 ? axis_class(k, g.n) : 1;
  v.cls = v.c[0] + 3 * v.c[1] + (D == 3 ? 9 * v.c[2] : 0);
  return true;
}
template <int D>
__device__ __forceinline__ bool vertex_of_thread(const Geom& g, Vtx<D>& v) {
  return vertex_of_thread_at<D>(g, D == 3 ? (int)blockIdx.z : 0, v);
}
// batched grid (x, 1, (D == 3 ? n1 : 1) * count): problem index and z-plane
template <int D>
__device__ __forceinline__ int batch_problem(const Geom& g) {
  return D == 3 ? (int)blockIdx.z / g.n1 : (int)blockIdx.z;
}
template <int D>
__device__ __forceinline__ int batch_plane(const Geom& g) {
  return D == 3 ? (int)blockIdx.z % g.n1 : 0;
}

// Is the neighbour at offset O inside the domain?
template <int D, int O>
__device__ __forceinline__ bool nb_valid(const int c[3]) {
  bool ok = true;
  static_for<0, D>([&](auto A) {
    constexpr int s = off_comp(D, O, decltype(A)::value);
    if constexpr (s == 1) ok = ok && (c[decltype(A)::value] != 2);
    if constexpr (s == -1) ok = ok && (c[decltype(A)::value] != 0);
  });
  return ok;
}
template <int D, int O>
__device__ __forceinline__ long long nb_delta(const Geom& g) {
  return (long long)off_comp(D, O, 0) + g.sy * off_comp(D, O, 1) +
         (D == 3 ? g.sz * off_comp(D, O, 2) : 0);
}
// Does the cell of incidence I exist for a vertex of this class?
template <int D, int I>
__device__ __forceinline__ bool inc_valid(const int c[3]) {
  bool ok = true;
  static_for<0, D>([&](auto A) {
    constexpr int a = decltype(A)::value;
    constexpr bool neg = (inc_corner(D, I) >> a) & 1;
    ok = ok && (neg ? c[a] != 0 : c[a] != 2);
  });
  return ok;
}

template <typename T> __device__ __forceinline__ double to_d(T x) { return (double)x; }
template <> __device__ __forceinline__ double to_d<__half>(__half x) { return (double)__half2float(x); }
template <typename T> __device__ __forceinline__ T from_d(double x) { return (T)x; }
template <> __device__ __forceinline__ __half from_d<__half>(double x) { return __float2half((float)x); }

// float -> double by integer operations only (exact; zeros, infinities, NaNs
// and subnormals included).  The hardware conversion runs on the float64 pipe,
// which bounds the float64 kernels that widen float32 inputs.
__device__ __forceinline__ double f2d_exact(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned m = u & 0x7fffffu;
  const unsigned long long sgn = (unsigned long long)(u & 0x80000000u) << 32;
  unsigned long long ex, mm;
  if (e != 0u) {                       // normal (rebias the exponent), or inf / NaN
    ex = e == 0xffu ? 0x7ffull : (unsigned long long)(e + 896u);
    mm = (unsigned long long)m << 29;
  } else {                             // zero, or subnormal m 2^-149: normalise
    const int p = 31 - __clz(m | 1u);  // leading one of m
    ex = m ? (unsigned long long)(p + 874) : 0ull;
    mm = m ? (((unsigned long long)m << (52 - p)) & 0xfffffffffffffull) : 0ull;
  }
  return __longlong_as_double((long long)(sgn | (ex << 52) | mm));
}

// Load all NOFF neighbour values of x (zero outside the domain).
template <int D, typename TX, typename T>
__device__ __forceinline__ void load_nb(const TX* __restrict__ x, const Geom& g, const Vtx<D>& v,
                                        T out[Topo<D>::NOFF]) {
  static_for<0, Topo<D>::NOFF>([&](auto O) {
    constexpr int o = decltype(O)::value;
    out[o] = nb_valid<D, o>(v.c) ? (T)x[v.idx + nb_delta<D, o>(g)] : (T)0;
  });
}

// sum_o W[cls][o] x_o over the first NO offsets (NOFF for M-like, NAX for K)
template <int D, int NO, typename T>
__device__ __forceinline__ T dot_w(const T* __restrict__ W, int cls, const T xs[]) {
  const T* w = W + cls * Topo<D>::NOFF;
  T acc = w[0] * xs[0];
#pragma unroll
  for (int o = 1; o < NO; ++o) acc = fma(w[o], xs[o], acc);
  return acc;
}

// ---------------------------------------------------------------------------
// per-level operator tables (device memory) and host-side bookkeeping
// ---------------------------------------------------------------------------
// Table layout: W[cls * NOFF + o], one table per operator per level.
template <typename T> struct OpTables {
  const T* M;      // mass weights of the level
  const T* K;      // stiffness weights
  const T* S;      // S_hat = M + gamma K
  const T* dinvM;  // 1 / diag(M) per class
  const T* dinvS;  // 1 / diag(S_hat) per class
};

// Host: reference (h = 1) tables of M and K for every class, double.
// WM[cls*NOFF+o] * h^d and WK[cls*NOFF+o] * h^(d-2) are the assembled weights.
void reference_tables(int dim, double* WM, double* WK);

// Batched launches (ok_solve_batch's cohorts): the arguments of up to
// BATCH_MAX independent problems travel by value in the kernel parameters;
// blockIdx.y (or a folded blockIdx.z) selects the problem.
constexpr int BATCH_MAX = 8;
template <typename A> struct Batch {
  A a[BATCH_MAX];
};

// reduction scratch layout helpers
constexpr int RED_MAX_BLOCKS = 1024;
constexpr int KRYLOV_MAX = 64;   // basis vectors per multi-dot (restart <= 63)

}  // namespace okg
