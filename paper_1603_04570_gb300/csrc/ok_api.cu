// ok_api.cu -- the C ABI (include/ok.h): grid handles, the preconditioner,
// flexible GMRES, Newton and the theta-method timestep.
//
// Host code here only sequences kernels and moves scalars; every arithmetic
// step of the solve runs in the kernels of ok_fem.cu, ok_mg.cu, ok_krylov.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "../../include/ok.h"
#include "ok_internal.cuh"
#include "ok_kernels.h"

using namespace okg;

namespace {

thread_local std::string g_last_error;

struct OkError {
  int status;
  std::string msg;
};

[[noreturn]] void fail(int status, const std::string& msg) { throw OkError{status, msg}; }

void ck(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    if (e == cudaErrorMemoryAllocation) {
      cudaGetLastError();
      fail(OK_ERR_NOMEM, std::string(what) + ": " + cudaGetErrorString(e));
    }
    fail(OK_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  }
}
#define CK(call) ck((call), #call)
#define CKL() ck(cudaGetLastError(), "kernel launch")

template <typename F>
int guarded(F&& f) {
  try {
    f();
    g_last_error.clear();
    return OK_SUCCESS;
  } catch (const OkError& e) {
    g_last_error = e.msg;
    return e.status;
  } catch (const std::bad_alloc&) {
    g_last_error = "host allocation failed";
    return OK_ERR_NOMEM;
  } catch (const std::exception& e) {
    g_last_error = std::string("internal error: ") + e.what();
    return OK_ERR_INTERNAL;
  } catch (...) {
    g_last_error = "internal error";
    return OK_ERR_INTERNAL;
  }
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void cheb_coefs(double lo, double hi, int steps, std::vector<double>& c1, std::vector<double>& c2, double& th) {
  th = 0.5 * (hi + lo);
  const double de = 0.5 * (hi - lo);
  double rho = de / th;
  c1.assign(steps > 1 ? steps - 1 : 1, 0.0);
  c2.assign(steps > 1 ? steps - 1 : 1, 0.0);
  for (int k = 0; k + 1 < steps; ++k) {
    const double rn = 1.0 / (2.0 * th / de - rho);
    c1[k] = rn * rho;
    c2[k] = 2.0 * rn / de;
    rho = rn;
  }
}

}  // namespace

std::atomic<long long> okg::g_launch_count{0};
thread_local bool okg::g_pdl = false;

// ---------------------------------------------------------------------------
// sampled kernel timing: one CUDA-event pair per kernel class per Arnoldi
// step, recorded on the handle's stream (inside the captured graph when
// graphs are on) and read after the step's host synchronisation.
// ---------------------------------------------------------------------------
enum ProfTag {
  PT_PRECOND = 0, PT_APPLYJ, PT_CGS2, PT_SMOOTH0, PT_CHEBM, PT_TPRE0, PT_TPOST0, PT_TAMASS,
  PT_TPRE1, PT_TPOST1, PT_TPRE2, PT_TPOST2, PT_TPRE3, PT_TPOST3, PT_TPRE4, PT_TPOST4, PT_COARSE, PT_LOW, PT_COUNT
};
static const char* const kProfNames[PT_COUNT] = {
    "precond", "apply_j", "cgs2", "mg_smooth_l0", "cheb_mass_step", "mg_tile_pre_l0", "mg_tile_post_l0",
    "tile_mass_cstep", "mg_tile_pre_l1", "mg_tile_post_l1", "mg_tile_pre_l2", "mg_tile_post_l2",
    "mg_tile_pre_l3", "mg_tile_post_l3", "mg_tile_pre_l4", "mg_tile_post_l4", "mg_coarse", "mg_low"};
// tags of the tile kernels of level l (pre, post); -1 below level 4
static inline int tile_tag(int l, bool post) {
  if (l == 0) return post ? PT_TPOST0 : PT_TPRE0;
  if (l <= 4) return PT_TPRE1 + 2 * (l - 1) + (post ? 1 : 0);
  return -1;
}
using TagSet = std::array<bool, PT_COUNT>;

struct Profiler {
  bool on = false;
  cudaEvent_t ev[PT_COUNT][2] = {};
  TagSet began{}, ended{};
  long long samples[PT_COUNT] = {};
  double total_ms[PT_COUNT] = {};
  void create() {
    for (int t = 0; t < PT_COUNT; ++t)
      for (int k = 0; k < 2; ++k)
        if (!ev[t][k]) CK(cudaEventCreate(&ev[t][k]));
  }
  void destroy() {
    for (int t = 0; t < PT_COUNT; ++t)
      for (int k = 0; k < 2; ++k)
        if (ev[t][k]) cudaEventDestroy(ev[t][k]), ev[t][k] = nullptr;
  }
  void reset_step() {
    began.fill(false);
    ended.fill(false);
  }
  void begin(int t, cudaStream_t s) {
    if (!on || t < 0 || began[t]) return;
    // "external" records stay real event records (timable) inside stream capture
    CK(cudaEventRecordWithFlags(ev[t][0], s, cudaEventRecordExternal));
    began[t] = true;
  }
  void end(int t, cudaStream_t s) {
    if (!on || t < 0 || !began[t] || ended[t]) return;
    CK(cudaEventRecordWithFlags(ev[t][1], s, cudaEventRecordExternal));
    ended[t] = true;
  }
  // after the stream was synchronised; a sample that cannot be read is skipped
  void collect(const TagSet& had) {
    for (int t = 0; t < PT_COUNT; ++t)
      if (had[t]) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ev[t][0], ev[t][1]) != cudaSuccess) {
          cudaGetLastError();
          continue;
        }
        samples[t] += 1;
        total_ms[t] += ms;
      }
  }
};

// ---------------------------------------------------------------------------
// device memory owned by a handle
// ---------------------------------------------------------------------------
// While ok_serve runs, the device blocks of destroyed handles are kept per
// (device, size) and handed to later handles that ask for the same sizes
// (requests of one grid and options ask for identical lists), so admitting a
// request does not call cudaMalloc / cudaFree next to the requests in flight;
// the blocks are freed when the last ok_serve returns.
struct DevicePool {
  std::mutex mu;
  int users = 0;
  std::multimap<std::pair<int, size_t>, void*> blocks;
};
DevicePool g_pool;

struct PoolScope {                    // pooling on for the lifetime of an ok_serve call
  PoolScope() {
    std::lock_guard<std::mutex> lk(g_pool.mu);
    ++g_pool.users;
  }
  ~PoolScope() {
    std::lock_guard<std::mutex> lk(g_pool.mu);
    if (--g_pool.users == 0) {
      for (auto& kv : g_pool.blocks) {
        int cur = 0;
        cudaGetDevice(&cur);
        cudaSetDevice(kv.first.first);
        cudaFree(kv.second);
        cudaSetDevice(cur);
      }
      g_pool.blocks.clear();
    }
  }
};

struct Arena {
  struct Block {
    void* p;
    size_t bytes;
    int device;
  };
  std::vector<Block> blocks;
  size_t bytes = 0;
  template <typename T>
  T* alloc(size_t count) {
    size_t b = count * sizeof(T);
    if (b == 0) b = 16;
    int dev = 0;
    cudaGetDevice(&dev);
    void* p = nullptr;
    {
      std::lock_guard<std::mutex> lk(g_pool.mu);
      auto it = g_pool.blocks.find({dev, b});
      if (it != g_pool.blocks.end()) {
        p = it->second;
        g_pool.blocks.erase(it);
      }
    }
    if (!p) {
      cudaError_t e = cudaMalloc(&p, b);
      if (e != cudaSuccess) {
        cudaGetLastError();
        fail(OK_ERR_NOMEM, "cudaMalloc of " + std::to_string(b) + " bytes failed: " + cudaGetErrorString(e));
      }
    }
    blocks.push_back({p, b, dev});
    bytes += b;
    return (T*)p;
  }
  void release() {
    std::lock_guard<std::mutex> lk(g_pool.mu);
    for (const Block& k : blocks) {
      if (g_pool.users > 0) {
        g_pool.blocks.insert({{k.device, k.bytes}, k.p});
      } else {
        int cur = 0;
        cudaGetDevice(&cur);
        if (cur != k.device) cudaSetDevice(k.device);
        cudaFree(k.p);
        if (cur != k.device) cudaSetDevice(cur);
      }
    }
    blocks.clear();
    bytes = 0;
  }
  ~Arena() { release(); }
};

// One multigrid level of S_hat in precision T.
template <typename T> struct Level {
  int n;
  Geom g;
  T *x, *b, *r, *d0, *d1;
  T* xa;           // second iterate buffer for the tile kernels (read one, write the other)
  T *WS, *dinvS;
};

// The block preconditioner in precision T (eqn prec with A~, S~).
template <typename T> struct Prec {
  int dim = 0;
  std::vector<Level<T>> lv;
  T *WM = nullptr, *WK = nullptr, *dinvM = nullptr;   // finest level M, K (scaled)
  T* coarse_inv = nullptr;
  long long nc = 0;
  T* gemv_inv = nullptr;       // nc > GEMV_MIN: the inverse with padded row stride gemv_ldA
  long long gemv_ldA = 0;
  static constexpr long long GEMV_MIN = 512;   // above: many-block GEMV, else one block
#ifndef OK_LOW_N1
#define OK_LOW_N1 129
#endif
  static constexpr int LOW_N1 = OK_LOW_N1;      // cluster kernel: levels of at most this many vertices per side

  // coarsest level above COARSE_NC_MAX unknowns (odd coarse sides such as the
  // 26^3 of n = 50 2^k): Chebyshev--Jacobi iteration from zero instead of the
  // dense inverse, qC steps on [lo, (d+2)/2] with lo = (1/2) / (1 + gamma rho),
  // rho = max over classes of diag(K)/diag(M) on that level (see build_prec)
  bool cheb_coarse = false;
  int qC = 0;
  double thC = 1;
  std::vector<double> cC1, cC2;
  void coarse_solve(const T* rhs, T* x, cudaStream_t s) {
    if (cheb_coarse) {
      Level<T>& C = lv.back();
      cheb<T, T>(C.g, C.WS, C.dinvS, rhs, true, x, C.r, C.d0, C.d1, qC, thC, cC1, cC2, (T*)nullptr, (T)1, false, s);
    } else if (gemv_inv) {
      launch_coarse_gemv<T>(nc, gemv_ldA, gemv_inv, rhs, x, s);
    } else {
      launch_coarse_solve<T>(nc, coarse_inv, rhs, x, s);
    }
  }
  T *cx = nullptr, *cr = nullptr, *cd0 = nullptr, *cd1 = nullptr;   // Chebyshev on M
  T *tt = nullptr, *yy = nullptr;                                    // k_R = 2
  const T* coef = nullptr;                                           // C coefficients (T)
  std::vector<double> cM1, cM2, cS1, cS2;
  double thM = 1, thS = 1;
  double inv_a11 = 1, dth = 0;
  int q_A = 10, n_V = 5, k_R = 1, nu_pre = 2, nu_post = 2;
  Profiler* prof = nullptr;
  bool fused = false;          // coarse levels Lc..L run as one shared-memory kernel
  int Lc = 0;
  CoarseArgs<T> ca{};
  CoarseArgs<T>* ca_dev = nullptr;   // device copy of ca (batched launches read it from there)
  size_t csmem = 0;
  bool low = false;            // 2D tiles: levels Lf.. and the coarsest solve in one cluster launch
  int Lf = 0, low_cluster = 0;
  LowArgs<T> la{};
  bool tiled = false;          // 2D: levels above Lc by shared-memory tile kernels
  std::vector<TileSmooth<T>> ts;
  TileMass<T> tm{};
  T* b2 = nullptr;             // right-hand side of the second S_hat solve (M S_hat^{-1} t)
  std::vector<int> cur;        // per level: 0 = x holds the iterate, 1 = xa does

  T* X(int l) { return cur[l] ? lv[l].xa : lv[l].x; }
  T* Xalt(int l) { return cur[l] ? lv[l].x : lv[l].xa; }

  // V-cycle with tile kernels on the levels above Lc (x ping-pongs between x and xa)
  template <typename TO>
  void vcycle_t(int l, bool x_zero, const T* rhs, TO* out, T* mx, cudaStream_t s) {
    if (low && l == Lf) {               // x from zero on rhs = lv[Lf].b; result in lv[Lf].x
      if (prof) prof->begin(PT_LOW, s);
      launch_low_vcycle<T>(la, low_cluster, s);
      if (prof) prof->end(PT_LOW, s);
      return;
    }
    if (fused && l == Lc) {
      if (prof) prof->begin(PT_COARSE, s);
      launch_coarse_vcycle<T>(dim, ca, csmem, rhs, x_zero ? (const T*)nullptr : X(l), X(l), s);
      if (prof) prof->end(PT_COARSE, s);
      return;
    }
    if (l + 1 == (int)lv.size()) {
      if (prof) prof->begin(PT_COARSE, s);
      coarse_solve(rhs, X(l), s);
      if (prof) prof->end(PT_COARSE, s);
      return;
    }
    if (prof) prof->begin(tile_tag(l, false), s);
    launch_tile_pre<T>(ts[l], x_zero ? (const T*)nullptr : X(l), rhs, Xalt(l), lv[l + 1].b, s);
    if (prof) prof->end(tile_tag(l, false), s);
    cur[l] ^= 1;
    vcycle_t<T>(l + 1, true, lv[l + 1].b, (T*)nullptr, (T*)nullptr, s);
    if (prof) prof->begin(tile_tag(l, true), s);
    launch_tile_post<T, TO>(ts[l], X(l), X(l + 1), rhs, Xalt(l), mx, out, (T)1, s);
    if (prof) prof->end(tile_tag(l, true), s);
    cur[l] ^= 1;
  }

  template <typename TO>
  void mg_solve_t(const T* rhs, TO* out, T* mx, cudaStream_t s) {
    std::fill(cur.begin(), cur.end(), 0);
    for (int c = 0; c < n_V; ++c) {
      const bool last = c + 1 == n_V;
      vcycle_t<TO>(0, c == 0, rhs, last ? out : (TO*)nullptr, last ? mx : (T*)nullptr, s);
    }
  }

  template <typename TZ>
  void apply_tiled(const double* v, TZ* z, cudaStream_t s) {
    const long long nv = lv[0].g.nv;
    if (prof) prof->begin(PT_TAMASS, s);
    launch_tile_amass<T, TZ>(tm, v, z, lv[0].b, s);            // z1 = A~^{-1} r1, t = r2 - C z1
    if (prof) prof->end(PT_TAMASS, s);
    mg_solve_t<T>(lv[0].b, (T*)nullptr, b2, s);                  // b2 = M S_hat^{-1} t
    mg_solve_t<TZ>(b2, z + nv, (T*)nullptr, s);                  // z2 = S_hat^{-1} b2
  }

  bool plane3 = false;         // 3D: stencil steps by z-marching blocks (ok_plane3.cu)
  std::vector<int> pshape;     // per level: block shape of the z-marching kernels
  std::vector<std::pair<int, int>> tuned;   // (cells per side, choice) the autotuner recorded
  int plane_shape(const Geom& g) const {
    for (size_t l = 0; l < lv.size(); ++l)
      if (lv[l].g.n == g.n) return l < pshape.size() ? pshape[l] : 0;
    return 0;
  }
  // the z-marching kernels on level g (shape PLANE_SHAPES: the autotuner found
  // the one-thread-per-vertex kernels faster there)
  bool on_planes(const Geom& g) const { return plane3 && plane_shape(g) < PLANE_SHAPES; }

  // out = n_V V-cycles from zero on the level-0 system with right-hand side rhs
  void solve_mg(const T* rhs, T* out, cudaStream_t s) {
    if (tiled) {
      mg_solve_t<T>(rhs, out, (T*)nullptr, s);
    } else {
      launch_axpby<T, T>(lv[0].g.nv, 1.0, rhs, 0.0, lv[0].b, s);
      mg_solve<T>(out, s);
    }
  }

  template <typename TB, typename TO>
  void cheb(const Geom& g, const T* W, const T* dinv, const TB* b, bool x_zero, T* x, T* r, T* d0, T* d1,
            int steps, double th, const std::vector<double>& c1, const std::vector<double>& c2, TO* out,
            T oscale, bool want_r, cudaStream_t s, int tag = -1, bool inited = false,
            const T** defer_last = nullptr) {
    // inited: the start from zero (r, d0) was written by the restriction
    // launch; defer_last: the last step (x += d, no residual, no output) is
    // left to the prolongation that reads x next, which gets d here
    if (x_zero) {
      if (!inited) launch_cheb_init<T, TB>(dim, g, dinv, b, (T)1, r, d0, (T)(1.0 / th), s);
    } else if (on_planes(g)) launch_resid_init3<T>(g, W, dinv, (const T*)b, x, r, d0, (T)(1.0 / th), s, plane_shape(g));
    else launch_resid_init<T>(dim, g, W, dinv, (const T*)b, x, r, d0, (T)(1.0 / th), s);
    T* d[2] = {d0, d1};
    int cur = 0;
    for (int k = 0; k + 1 < steps; ++k) {
      if (k == 0 && prof) prof->begin(tag, s);
      if (on_planes(g))
        launch_cheb_step3<T>(g, W, dinv, x, r, d[cur], d[1 - cur], (T)c1[k], (T)c2[k], x_zero && k == 0, s,
                             plane_shape(g));
      else
        launch_cheb_step<T>(dim, g, W, dinv, x, r, d[cur], d[1 - cur], (T)c1[k], (T)c2[k], x_zero && k == 0, s);
      if (k == 0 && prof) prof->end(tag, s);
      cur ^= 1;
    }
    if (defer_last && !want_r && out == nullptr && !(x_zero && steps == 1)) {
      *defer_last = d[cur];
      return;
    }
    if (on_planes(g) && want_r)
      launch_cheb_last3<T, TO>(g, W, x, r, d[cur], x_zero && steps == 1, out, oscale, s, plane_shape(g));
    else launch_cheb_last<T, TO>(dim, g, W, x, want_r ? r : nullptr, d[cur], x_zero && steps == 1, out, oscale, s);
  }
  // y = alpha W x on level g (M x, or dt theta K y for k_R = 2)
  void op(const Geom& g, const T* W, bool axis_only, const T* x, T* y, T alpha, cudaStream_t s) {
    if (on_planes(g))
      launch_op_apply3<T, T, T>(g, W, axis_only, x, y, alpha, (const T*)nullptr, (T)0, s, plane_shape(g));
    else launch_op_apply<T, T, T>(dim, g, W, axis_only, x, y, alpha, (const T*)nullptr, (T)0, s);
  }

  // inited / defer: see cheb (level l's start from zero was written by the
  // restriction above it; its last post-smoothing step goes to the caller's
  // prolongation)
  template <typename TO>
  void vcycle(int l, bool x_zero, TO* out, cudaStream_t s, bool inited = false, const T** defer = nullptr) {
    Level<T>& L = lv[l];
    const bool coarsest = (l + 1 == (int)lv.size());
    if (fused && l == Lc) {                 // levels Lc..L in one thread block
      launch_coarse_vcycle<T>(dim, ca, csmem, L.b, x_zero ? (const T*)nullptr : L.x, L.x, s);
      if (out) launch_axpby<T, TO>(L.g.nv, 1.0, L.x, 0.0, out, s);
      return;
    }
    if (coarsest) {
      coarse_solve(L.b, L.x, s);
      if (out) launch_axpby<T, TO>(L.g.nv, 1.0, L.x, 0.0, out, s);
      return;
    }
    cheb<T, T>(L.g, L.WS, L.dinvS, L.b, x_zero, L.x, L.r, L.d0, L.d1, nu_pre, thS, cS1, cS2, (T*)nullptr,
               (T)1, true, s, l == 0 ? PT_SMOOTH0 : -1, inited);
    Level<T>& C = lv[l + 1];
    // a coarse level that smooths (neither the fused part nor the coarsest)
    // starts inside the restriction launch and ends inside the prolongation
    const bool c_smooths = !(fused && l + 1 == Lc) && l + 2 < (int)lv.size();
    if (c_smooths) launch_restrict<T>(dim, L.g, C.g, L.r, C.b, s, C.dinvS, C.r, C.d0, (T)(1.0 / thS));
    else launch_restrict<T>(dim, L.g, C.g, L.r, C.b, s);
    const T* dc = nullptr;
    vcycle<T>(l + 1, true, (T*)nullptr, s, c_smooths, c_smooths ? &dc : nullptr);
    launch_prolong_add<T>(dim, L.g, C.g, L.x, C.x, s, dc);
    cheb<T, TO>(L.g, L.WS, L.dinvS, L.b, false, L.x, L.r, L.d0, L.d1, nu_post, thS, cS1, cS2, out, (T)1, false, s,
                -1, false, defer);
  }

  // x_0 = S_hat^{-1} b_0 by n_V V-cycles from zero; optional cast to out
  template <typename TO>
  void mg_solve(TO* out, cudaStream_t s) {
    for (int c = 0; c < n_V; ++c) vcycle<TO>(0, c == 0, c + 1 == n_V ? out : (TO*)nullptr, s);
  }

  // A~^{-1} b into cx (unscaled Chebyshev on M; A~^{-1} b = cx / a11)
  template <typename TB, typename TO>
  void a_inv(const TB* b, TO* out, cudaStream_t s) {
    cheb<TB, TO>(lv[0].g, WM, dinvM, b, true, cx, cr, cd0, cd1, q_A, thM, cM1, cM2, out, (T)inv_a11, false, s,
                 PT_CHEBM);
  }

  // z = P^{-1} v  (v: 2 nv doubles; z: 2 nv of TZ)
  template <typename TZ>
  void apply(const double* v, TZ* z, cudaStream_t s) {
    if (tiled) {
      apply_tiled<TZ>(v, z, s);
      return;
    }
    const Geom& g = lv[0].g;
    const long long nv = g.nv;
    Level<T>& L0 = lv[0];
    a_inv<double, TZ>(v, z, s);                                           // z1 = A~^{-1} r1
    launch_cstep<T, double>(dim, g, coef, v + nv, (T)1, cx, (T)inv_a11, L0.b, s);   // t = r2 - C z1
    if (k_R == 1) {
      mg_solve<T>((T*)nullptr, s);                                         // S_hat^{-1} t
      op(g, WM, false, L0.x, L0.b, (T)1, s);                               // M .
      mg_solve<TZ>(z + nv, s);                                             // S_hat^{-1} .
      return;
    }
    // k_R = 2: y = S~^{-1} t;  z2 = y + S~^{-1} (t - S y),  S y = M y - C A~^{-1} (dt theta K y)
    launch_axpby<T, T>(nv, 1.0, L0.b, 0.0, tt, s);
    mg_solve<T>((T*)nullptr, s);
    op(g, WM, false, L0.x, L0.b, (T)1, s);
    mg_solve<T>(yy, s);
    op(g, WK, true, yy, cr, (T)dth, s);                                                     // q = dt th K y
    launch_axpby<T, T>(nv, 1.0, cr, 0.0, L0.r, s);                                          // keep q
    a_inv<T, T>(L0.r, (T*)nullptr, s);                                                     // cx = Cheb(q)
    launch_schur_resid<T>(dim, g, WM, (T)1, coef, tt, yy, cx, (T)inv_a11, L0.b, s);         // t - S y
    mg_solve<T>((T*)nullptr, s);
    op(g, WM, false, L0.x, L0.b, (T)1, s);
    mg_solve<T>((T*)nullptr, s);
    launch_axpby<T, T>(nv, 1.0, yy, 1.0, L0.x, s);
    launch_axpby<T, TZ>(nv, 1.0, L0.x, 0.0, z + nv, s);
  }
};

struct ok_grid {
  int dim = 0, n = 0;
  int device = 0;
  int sms = 1;           // streaming multiprocessors of the device
  Geom g0;
  ok_params p;
  ok_opts o;
  Arena arena;
  cudaStream_t s = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  ResidualCoefs rc;
  JCoefs jc;
  int n_levels = 0;
  // reference tables (h = 1), double
  double *refWM = nullptr, *refWK = nullptr;
  double *WM0d = nullptr, *dinvM0d = nullptr;   // finest M (scaled), double: w0 projection
  // state and work vectors (double)
  double *un = nullptr, *wn = nullptr, *uk = nullptr, *wk = nullptr;   // N_v each
  double *f = nullptr, *xs = nullptr, *rv = nullptr, *tmp = nullptr;  // 2 N_v each
  double* coef = nullptr;
  float* coef32 = nullptr;
  // Krylov
  double* V = nullptr;
  double* Zd = nullptr;
  float* Zf = nullptr;
  __half* Zh = nullptr;
  KrylovState* ks = nullptr;
  RedScratch rs;
  double* dsc = nullptr;      // device scalars
  int* dflag = nullptr;
  double* hpin = nullptr;     // pinned host scalars
  Prec<double> pd;
  Prec<float> pf;
  std::vector<cudaGraphExec_t> graphs;   // one Arnoldi step per j
  std::vector<cudaGraphExec_t> cgraphs;  // the same behind a device-side IF (batched launches)
  std::vector<long long> cgraph_kernels;
  bool cond_ok = true;                   // conditional graphs build on this device
  std::vector<long long> graph_kernels;  // kernels captured in each graph
  std::vector<TagSet> graph_tags;        // profiled kernel classes in each graph
  Profiler prof;
  double cheb_init_th = 1;
  std::vector<double> cI1, cI2;          // 60-step mass Chebyshev for w0
  struct EnergyWork* ew = nullptr;       // ok_energy's multigrid and vectors (first call)
};

// ok_energy: multigrid of M + K (float64) as the preconditioner of conjugate
// gradients for the Neumann problem K phi = M f, and the vectors of that solve.
struct EnergyWork {
  Prec<double> mg;
  double *ones = nullptr, *lm = nullptr, *f = nullptr, *b = nullptr, *x = nullptr, *r = nullptr, *z = nullptr,
         *p = nullptr, *q = nullptr, *e = nullptr;
  int last_its = 0;
};

namespace {

// ---------------------------------------------------------------------------
// autotuner: the tile width (2D register-strip kernels) or block shape (3D
// z-marching kernels) of each multigrid level, chosen by timing the level's
// kernels once per (device, dim, n, precision) and cached for the process.
// Every choice computes the same bits, so only the time depends on it.
// ---------------------------------------------------------------------------
std::mutex g_tune_mu;
std::map<std::array<int, 5>, int> g_tune;   // (device, dim, n, sizeof(T), 0) -> choice
std::mutex g_tune_run_mu;                   // one tuning at a time: concurrent setups of one
                                            // shape then find the first one's choices

template <typename F>
float time_launches(F&& launch, int reps) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  launch();
  launch();                                        // warm-up
  CK(cudaEventRecord(e0, 0));
  for (int k = 0; k < reps; ++k) launch();
  CK(cudaEventRecord(e1, 0));
  CK(cudaEventSynchronize(e1));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CKL();
  return ms / reps;
}

template <typename T>
void autotune(ok_grid* G, Prec<T>& P) {
  const int nl = (int)P.lv.size();
  P.pshape.assign(nl, G->o.tile_fine >= 4 ? G->o.tile_fine - 4 : 0);   // 3D: 4 + k forces shape k
  if (G->o.tile_fine != 1) return;
  std::lock_guard<std::mutex> run(g_tune_run_mu);
  auto cached = [&](int n, int& out) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find({G->device, G->dim, n, (int)sizeof(T), 0});
    if (it == g_tune.end()) return false;
    out = it->second;
    return true;
  };
  auto store = [&](int n, int v) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[{G->device, G->dim, n, (int)sizeof(T), 0}] = v;
  };
  if (P.tiled) {                                   // 2D: strip window shape per tiled level
    const int top = P.fused ? P.Lc : nl - 1;
    for (int l = 0; l < top && l + 1 < nl; ++l) {
      Level<T>& L = P.lv[l];
      Level<T>& C = P.lv[l + 1];
      int best = 0;
      if (!cached(L.n, best)) {
        T* fine[] = {L.x, L.xa, L.b};
        T* coarse[] = {C.b, C.x};
        for (T* v : fine) CK(cudaMemset(v, 0, L.g.nv * sizeof(T)));
        for (T* v : coarse) CK(cudaMemset(v, 0, C.g.nv * sizeof(T)));
        float tbest = 0.f;
        best = -1;
        for (int w = 0; w < STRIP_SHAPES; ++w) {
          TileSmooth<T> ts = P.ts[l];
          ts.tile = w;
          const float t = time_launches([&] {
            launch_tile_pre<T>(ts, (const T*)nullptr, L.b, L.xa, C.b, 0);
            launch_tile_post<T, T>(ts, L.xa, C.x, L.b, L.x, (T*)nullptr, (T*)nullptr, (T)1, 0);
          }, 5);
          if (best < 0 || t < tbest) best = w, tbest = t;
        }
        store(L.n, best);
      }
      P.ts[l].tile = best;
      P.tuned.push_back({L.n, best});
    }
  } else if (P.plane3) {                           // 3D: block shape per level of the z-marching kernels
    // the levels whose stencil steps run by z-marching blocks: the finest (the
    // mass solve and M apply run there) and every smoothed level above the
    // fused part, the coarsest only when it is solved by Chebyshev iteration
    const int top = P.fused ? P.Lc : nl;
    for (int l = 0; l < top; ++l) {
      Level<T>& L = P.lv[l];
      if (l > 0 && l + 1 == nl && !P.cheb_coarse) break;
      int best = -1;
      if (!cached(L.n, best)) {
        T* vs[] = {L.x, L.r, L.d0, L.d1};
        for (T* v : vs) CK(cudaMemset(v, 0, L.g.nv * sizeof(T)));
        float tbest = 0.f;
        for (int sh = 0; sh <= PLANE_SHAPES; ++sh) {   // the last candidate: one thread per vertex
          const float t = time_launches([&] {
            if (sh < PLANE_SHAPES)
              launch_cheb_step3<T>(L.g, L.WS, L.dinvS, L.x, L.r, L.d0, L.d1, (T)0.5, (T)0.5, false, 0, sh);
            else
              launch_cheb_step<T>(3, L.g, L.WS, L.dinvS, L.x, L.r, L.d0, L.d1, (T)0.5, (T)0.5, false, 0);
          }, 5);
          if (best < 0 || t < tbest) best = sh, tbest = t;
        }
        store(L.n, best);
      }
      P.pshape[l] = best;
      P.tuned.push_back({L.n, best});
    }
  }
}

// The multigrid hierarchy of M + gamma K (gamma < 0: S_hat's eps sqrt(c)) and
// the rest of the block preconditioner's workspace.
template <typename T>
void build_prec(ok_grid* G, Prec<T>& P, const std::vector<int>& sizes, const std::vector<double>& refM,
                const std::vector<double>& refK, double gamma_in = -1.0) {
  const int dim = G->dim;
  const int NOFF = dim == 2 ? Topo<2>::NOFF : Topo<3>::NOFF;
  const int NCLASS = dim == 2 ? Topo<2>::NCLASS : Topo<3>::NCLASS;
  const double gamma = gamma_in >= 0.0 ? gamma_in
                                       : G->p.eps * std::sqrt(G->p.dt * G->p.theta /
                                                              (1.0 + G->p.dt * G->p.theta * G->p.sigma));
  Arena& A = G->arena;
  P.dim = dim;
  P.q_A = G->o.q_A;
  P.n_V = G->o.n_V;
  P.k_R = G->o.k_R;
  P.nu_pre = G->o.smooth_pre;
  P.nu_post = G->o.smooth_post;
  P.inv_a11 = 1.0 / (1.0 + G->p.dt * G->p.theta * G->p.sigma);
  P.dth = G->p.dt * G->p.theta;
  P.plane3 = dim == 3 && G->o.tile_fine != 0;
  const double hiS = 0.5 * (dim + 2);
  cheb_coefs(G->o.smooth_lo_frac * hiS, hiS, std::max(P.nu_pre, P.nu_post), P.cS1, P.cS2, P.thS);
  cheb_coefs(0.5, 0.5 * (dim + 2), P.q_A, P.cM1, P.cM2, P.thM);
  std::vector<T> tab(NCLASS * NOFF), dv(NCLASS);
  auto upload = [&](const std::vector<T>& h) {
    T* d = A.alloc<T>(h.size());
    CK(cudaMemcpy(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    return d;
  };
  for (size_t l = 0; l < sizes.size(); ++l) {
    Level<T> L;
    L.n = sizes[l];
    L.g = make_geom(dim, L.n);
    const double h = 1.0 / L.n;
    const double hd = std::pow(h, dim), hk = std::pow(h, dim - 2);
    for (int i = 0; i < NCLASS * NOFF; ++i) tab[i] = (T)(hd * refM[i] + gamma * hk * refK[i]);
    for (int c = 0; c < NCLASS; ++c) dv[c] = (T)(1.0 / (hd * refM[c * NOFF] + gamma * hk * refK[c * NOFF]));
    L.WS = upload(tab);
    L.dinvS = upload(dv);
    const long long nv = L.g.nv;
    L.x = A.alloc<T>(nv);
    L.b = A.alloc<T>(nv);
    L.r = A.alloc<T>(nv);
    L.d0 = A.alloc<T>(nv);
    L.d1 = A.alloc<T>(nv);
    L.xa = A.alloc<T>(nv);
    if (l == 0) {
      for (int i = 0; i < NCLASS * NOFF; ++i) tab[i] = (T)(hd * refM[i]);
      for (int c = 0; c < NCLASS; ++c) dv[c] = (T)(1.0 / (hd * refM[c * NOFF]));
      P.WM = upload(tab);
      P.dinvM = upload(dv);
      for (int i = 0; i < NCLASS * NOFF; ++i) tab[i] = (T)(hk * refK[i]);
      P.WK = upload(tab);
    }
    P.lv.push_back(L);
  }
  const long long nv0 = P.lv[0].g.nv;
  P.cx = A.alloc<T>(nv0);
  P.cr = A.alloc<T>(nv0);
  P.cd0 = A.alloc<T>(nv0);
  P.cd1 = A.alloc<T>(nv0);
  if (P.k_R == 2) {
    P.tt = A.alloc<T>(nv0);
    P.yy = A.alloc<T>(nv0);
  }
  // coarsest level: dense S_hat and its inverse (float64 Gauss--Jordan on the
  // GPU) up to COARSE_NC_MAX unknowns, else a Chebyshev solve on that level
  Level<T>& C = P.lv.back();
  const long long nc = C.g.nv;
  P.nc = nc;
  const bool dense_coarse = nc <= COARSE_NC_MAX;
  if (!dense_coarse) {
    // D^{-1} S_hat with S_hat = M + gamma K, D = D_M + gamma D_K: x^T S_hat x >= x^T M x
    // >= (1/2) x^T D_M x (the element bound of the mass interval) and x^T D x <=
    // (1 + gamma rho) x^T D_M x, so its spectrum lies in [(1/2)/(1 + gamma rho), (d+2)/2]
    const double h = 1.0 / C.n, hd = std::pow(h, dim), hk = std::pow(h, dim - 2);
    double rho = 0.0;
    for (int c = 0; c < NCLASS; ++c) rho = std::max(rho, hk * refK[c * NOFF] / (hd * refM[c * NOFF]));
    const double lo = 0.5 / (1.0 + gamma * rho), hi = 0.5 * (dim + 2);
    const double kap = hi / lo, sig = (std::sqrt(kap) + 1.0) / (std::sqrt(kap) - 1.0);
    const double tol = std::is_same<T, double>::value ? 1e-13 : 1e-8;
    // Chebyshev error after q steps <= 2 / (sig^q + sig^-q) <= tol
    P.qC = std::max(2, (int)std::ceil(std::log(2.0 / tol) / std::log(sig)));
    cheb_coefs(lo, hi, P.qC, P.cC1, P.cC2, P.thC);
    P.cheb_coarse = true;
  }
  if (dense_coarse) {
    const double h = 1.0 / C.n, hd = std::pow(h, dim), hk = std::pow(h, dim - 2);
    std::vector<double> td(NCLASS * NOFF);
    for (int i = 0; i < NCLASS * NOFF; ++i) td[i] = hd * refM[i] + gamma * hk * refK[i];
    Arena setup;                       // released when this block ends
    double* Wd = setup.alloc<double>(td.size());
    CK(cudaMemcpy(Wd, td.data(), td.size() * sizeof(double), cudaMemcpyHostToDevice));
    double* dense = setup.alloc<double>(nc * nc);
    double* work = setup.alloc<double>(2 * nc * nc + nc);
    double* inv = std::is_same<T, double>::value ? A.alloc<double>(nc * nc) : setup.alloc<double>(nc * nc);
    CK(cudaMemset(dense, 0, nc * nc * sizeof(double)));
    launch_dense_from_table(dim, C.g, Wd, dense, 0);
    CKL();
    launch_gauss_jordan(nc, dense, work, inv, 0);
    CKL();
    if (std::is_same<T, double>::value) {
      P.coarse_inv = (T*)inv;
    } else {
      P.coarse_inv = A.alloc<T>(nc * nc);
      launch_axpby<double, T>(nc * nc, 1.0, inv, 0.0, P.coarse_inv, 0);
      CKL();
    }
    if (nc > P.GEMV_MIN) {           // padded copy for the many-block GEMV
      P.gemv_ldA = gemv_ld(nc, sizeof(T));
      P.gemv_inv = A.alloc<T>(nc * P.gemv_ldA);
      CK(cudaMemset(P.gemv_inv, 0, nc * P.gemv_ldA * sizeof(T)));
      CK(cudaMemcpy2D(P.gemv_inv, P.gemv_ldA * sizeof(T), P.coarse_inv, nc * sizeof(T), nc * sizeof(T), nc,
                      cudaMemcpyDeviceToDevice));
      CK(prepare_coarse_gemv<T>(nc));
    }
    CK(cudaStreamSynchronize(0));      // setup work of this handle (legacy stream); other handles keep running
  }
  // fused coarse part: the longest suffix of levels whose five vectors fit in
  // shared memory (at most COARSE_MAXLEV levels); worth it from two levels on
  const int nl = (int)P.lv.size();
  const size_t budget = COARSE_SMEM_MAX;
  // 2D tile kernels need two smoothing steps, the S~^{-1} form and the
  // ten-step mass solve they are compiled for (the paper's ten Chebyshev steps)
  const bool tiles_ok =
      G->o.tile_fine && dim == 2 && P.nu_pre == 2 && P.nu_post == 2 && P.k_R == 1 && P.q_A == 10;
  size_t tot = 0;
  int Lc = nl;
  for (int l = nl - 1; l >= 0; --l) {
    const size_t need = (5 * (size_t)P.lv[l].g.nv + NCLASS * NOFF + NCLASS) * sizeof(T);
    // one SM issues the whole fused part: keep its largest level small
    // (<= 1200 vertices, 33^2 in 2D, 9^3 in 3D) when a multi-block path exists
    // for the levels above it (the 2D tile kernels)
    const bool small_enough = P.lv[l].g.nv <= 1200 || !tiles_ok;
    if (tot + need > budget || nl - l > COARSE_MAXLEV || !small_enough) break;
    tot += need;
    Lc = l;
  }
  // fuse_coarse == 2 with the 2D tile kernels: the levels of at most LOW_N1
  // vertices per side (from level 1 down) and the coarsest solve run as one
  // thread-block cluster when the device supports it; otherwise (and with
  // fuse_coarse == 1) the single-block coarse V-cycle for the suffix above.
  // (On GB300 at 1025^2 the cluster launch is slower than separate launches:
  // 16 SMs leave most of each phase's windows serialised.)
  int low_cluster = 0, Lf = nl - 1;
  if (tiles_ok && G->o.fuse_coarse == 2 && nl >= 3 && dense_coarse) {
    for (int l = 1; l < nl - 1; ++l)
      if (P.lv[l].g.n1 <= Prec<T>::LOW_N1) {
        Lf = l;
        break;
      }
    const int nlow = nl - 1 - Lf;
    if (nlow >= 1 && nlow <= LOW_MAXLEV) low_cluster = prepare_low_vcycle<T>(nc);
  }
  if (G->o.fuse_coarse && low_cluster == 0 && nl - Lc >= 2 && dense_coarse) {
    CoarseArgs<T>& ca = P.ca;
    ca.nlev = nl - Lc;
    long long off = 0;
    for (int i = 0; i < ca.nlev; ++i) {
      const Level<T>& L = P.lv[Lc + i];
      ca.g[i] = L.g;
      ca.W[i] = L.WS;
      ca.dinv[i] = L.dinvS;
      ca.off[i] = off;
      off += 5 * L.g.nv;
      ca.mul[i] = (unsigned)((0x100000000ull + L.g.n1 - 1) / L.g.n1);   // ceil(2^32 / (n+1))
      const unsigned long long wI = L.g.n > 2 ? (unsigned long long)(L.g.n - 1) : 2ull;
      ca.mulI[i] = (unsigned)((0x100000000ull + wI - 1) / wI);           // ceil(2^32 / (n-1))
    }
    for (int i = 0; i < ca.nlev; ++i) {          // table copies after the vectors
      ca.toff[i] = off;
      off += NCLASS * NOFF + NCLASS;
    }
    ca.Ainv = P.coarse_inv;
    ca.inv_th = (T)(1.0 / P.thS);
    for (int k = 0; k < 16; ++k) {
      ca.c1[k] = k < (int)P.cS1.size() ? (T)P.cS1[k] : (T)0;
      ca.c2[k] = k < (int)P.cS2.size() ? (T)P.cS2[k] : (T)0;
    }
    ca.nu_pre = P.nu_pre;
    ca.nu_post = P.nu_post;
    P.csmem = (size_t)off * sizeof(T);
    CK(prepare_coarse_vcycle<T>(dim, P.csmem));
    P.ca_dev = (CoarseArgs<T>*)A.alloc<char>(sizeof(CoarseArgs<T>));
    CK(cudaMemcpy(P.ca_dev, &P.ca, sizeof(CoarseArgs<T>), cudaMemcpyHostToDevice));
    P.fused = true;
    P.Lc = Lc;
  }
  P.cur.assign(nl, 0);
  // 2D tile kernels for the levels above the fused part (two smoothing steps,
  // S~^{-1} form, at most 16 mass Chebyshev steps)
  const int top = P.fused ? P.Lc : nl - 1;
  // (the mass kernel is compiled for q_A = 10, the paper's ten Chebyshev steps)
  if (tiles_ok && top >= 1) {
    P.ts.resize(nl);
    for (int l = 0; l + 1 < nl; ++l) {
      TileSmooth<T>& t = P.ts[l];
      t.g = P.lv[l].g;
      t.gc = P.lv[l + 1].g;
      t.W = P.lv[l].WS;
      t.dinv = P.lv[l].dinvS;
      t.WM = P.WM;            // only used on level 0 (M x between the two S_hat solves)
      t.inv_th = (T)(1.0 / P.thS);
      t.c1 = (T)P.cS1[0];
      t.c2 = (T)P.cS2[0];
      // 64-column windows on levels of at least 1000 vertices per side (less
      // redundant halo work), 32-column windows below (more, shorter blocks;
      // measured faster from 513^2 down); tile_fine = 2 or 3 forces 32 or 64
      // on every tiled level
      const int tf = G->o.tile_fine;
      t.tile = tf == 2 ? 0 : (tf == 3 ? 1 : (t.g.n1 >= 1000 ? 1 : 0));   // shape (autotuned when tf == 1)
    }
    TileMass<T>& m = P.tm;
    m.g = P.lv[0].g;
    m.WM = P.WM;
    m.dinvM = P.dinvM;
    m.coef = nullptr;         // set when the coefficient store is bound
    m.sx = P.cx;              // the Chebyshev-on-M buffers of the untiled path
    m.sr = P.cr;
    m.sd = P.cd0;
    m.q = P.q_A;
    m.inv_th = (T)(1.0 / P.thM);
    m.inv_a11 = (T)P.inv_a11;
    for (int k = 0; k < 16; ++k) {
      m.c1[k] = k < (int)P.cM1.size() ? (T)P.cM1[k] : (T)0;
      m.c2[k] = k < (int)P.cM2.size() ? (T)P.cM2[k] : (T)0;
    }
    P.b2 = A.alloc<T>(P.lv[0].g.nv);
    CK(prepare_tiles<T>(P.q_A));
    P.tiled = true;
    if (low_cluster > 0) {
      LowArgs<T>& la = P.la;
      la.nl = nl - 1 - Lf;
      for (int i = 0; i < la.nl; ++i) {
        la.ts[i] = P.ts[Lf + i];
        la.P[i] = P.lv[Lf + i].xa;       // the iterate buffers never swap below Lf (x from zero, two
        la.Q[i] = P.lv[Lf + i].x;        // swaps per V-cycle), so the launch arguments are fixed
        la.rhs[i] = P.lv[Lf + i].b;
      }
      la.rhs[la.nl] = P.lv[nl - 1].b;
      la.xc = P.lv[nl - 1].x;
      if (!P.gemv_inv) {
        P.gemv_ldA = gemv_ld(nc, sizeof(T));
        P.gemv_inv = A.alloc<T>(nc * P.gemv_ldA);
        CK(cudaMemset(P.gemv_inv, 0, nc * P.gemv_ldA * sizeof(T)));
        CK(cudaMemcpy2D(P.gemv_inv, P.gemv_ldA * sizeof(T), P.coarse_inv, nc * sizeof(T), nc * sizeof(T), nc,
                        cudaMemcpyDeviceToDevice));
      }
      la.nc = nc;
      la.ldA = P.gemv_ldA;
      la.A = P.gemv_inv;
      P.low = true;
      P.Lf = Lf;
      P.low_cluster = low_cluster;
    }
  }
  autotune<T>(G, P);
  CK(cudaStreamSynchronize(0));
}

void validate(int dim, int n, const ok_params* p, const ok_opts* o) {
  if (dim != 2 && dim != 3) fail(OK_ERR_INVALID_ARG, "dim must be 2 or 3");
  if (n < 2) fail(OK_ERR_INVALID_ARG, "n must be >= 2");
  double nv = std::pow((double)(n + 1), dim);
  if (nv >= 2147483647.0) fail(OK_ERR_INVALID_ARG, "(n+1)^dim must be < 2^31");
  if (!p) fail(OK_ERR_INVALID_ARG, "params is NULL");
  if (!(p->eps > 0) || !(p->dt > 0) || !(p->theta > 0 && p->theta <= 1) || !(p->sigma >= 0) ||
      !std::isfinite(p->m) || !std::isfinite(p->eps) || !std::isfinite(p->dt) || !std::isfinite(p->sigma))
    fail(OK_ERR_INVALID_ARG, "params out of range (need eps > 0, dt > 0, 0 < theta <= 1, sigma >= 0)");
  if (o->restart < 1 || o->restart >= KRYLOV_MAX) fail(OK_ERR_INVALID_ARG, "restart must be in [1, 63]");
  if (o->q_A < 1 || o->n_V < 1 || o->smooth_pre < 1 || o->smooth_post < 1 || o->q_A > 64 || o->smooth_pre > 16 ||
      o->smooth_post > 16 || o->n_V > 32)
    fail(OK_ERR_INVALID_ARG, "q_A, n_V, smooth_pre, smooth_post must be >= 1 (and q_A <= 64, n_V <= 32, smoothing <= 16)");
  if (o->k_R != 1 && o->k_R != 2) fail(OK_ERR_INVALID_ARG, "k_R must be 1 or 2");
  if (o->precision != OK_FP64 && o->precision != OK_MIXED && o->precision != OK_MIXED_HALF)
    fail(OK_ERR_INVALID_ARG, "precision must be OK_FP64, OK_MIXED or OK_MIXED_HALF");
  if (o->max_gmres < 1 || o->max_newton < 0 || o->newton_extra < 0) fail(OK_ERR_INVALID_ARG, "iteration caps");
  if (!(o->gmres_rtol > 0) || !(o->newton_atol >= 0) || !(o->newton_rtol >= 0))
    fail(OK_ERR_INVALID_ARG, "tolerances must be positive");
  if (!(o->smooth_lo_frac > 0 && o->smooth_lo_frac < 1)) fail(OK_ERR_INVALID_ARG, "smooth_lo_frac in (0,1)");
  if (o->coarse_max < 1) fail(OK_ERR_INVALID_ARG, "coarse_max must be >= 1");
  if (o->tile_fine < 0 || o->tile_fine > (dim == 3 ? 7 : 3))
    fail(OK_ERR_INVALID_ARG, "tile_fine must be 0, 1, 2 or 3 (3D: also 4..7)");
  if (o->reorth < 0 || o->reorth > 2) fail(OK_ERR_INVALID_ARG, "reorth must be 0, 1 or 2");
  if (o->fuse_coarse < 0 || o->fuse_coarse > 2) fail(OK_ERR_INVALID_ARG, "fuse_coarse must be 0, 1 or 2");
}

std::vector<int> level_sizes(int n, int coarse_max) {
  std::vector<int> s{n};
  while (s.back() % 2 == 0 && s.back() > coarse_max) s.push_back(s.back() / 2);
  return s;
}

struct StreamScope {
  ok_grid* G;
  cudaStream_t user;
  StreamScope(ok_grid* g, cudaStream_t u) : G(g), user(u) {
    g_pdl = G->o.use_pdl != 0;
    CK(cudaEventRecord(G->ev_in, user));
    CK(cudaStreamWaitEvent(G->s, G->ev_in, 0));
  }
  ~StreamScope() {
    if (cudaEventRecord(G->ev_out, G->s) == cudaSuccess) cudaStreamWaitEvent(user, G->ev_out, 0);
  }
};

// bring a caller array into device memory (copy if it is on the host)
const double* stage_in(ok_grid* G, const double* p, double* buf, long long count) {
  if (!p) fail(OK_ERR_INVALID_ARG, "NULL array");
  if (is_device_ptr(p)) return p;
  CK(cudaMemcpyAsync(buf, p, count * sizeof(double), cudaMemcpyHostToDevice, G->s));
  return buf;
}

void check_finite(ok_grid* G, const double* d, long long count, const char* what) {
  CK(cudaMemsetAsync(G->dflag, 0, sizeof(int), G->s));
  launch_check_finite(d, count, G->dflag, G->s);
  CKL();
  int h = 0;
  CK(cudaMemcpyAsync(G->hpin, G->dflag, sizeof(int), cudaMemcpyDeviceToHost, G->s));
  CK(cudaStreamSynchronize(G->s));
  std::memcpy(&h, G->hpin, sizeof(int));
  if (h) fail(OK_ERR_NONFINITE, std::string("non-finite value in ") + what);
}

double read_scalar(ok_grid* G, const double* d) {
  CK(cudaMemcpyAsync(G->hpin, d, sizeof(double), cudaMemcpyDeviceToHost, G->s));
  CK(cudaStreamSynchronize(G->s));
  return G->hpin[0];
}

void assemble_c(ok_grid* G, const double* uk) {
  launch_assemble_c(G->dim, G->g0, G->rc, uk, G->coef, G->coef32, G->s);
  CKL();
}

// z = P^{-1} v with the configured precision (z: 2 nv, Z-slot type)
template <typename TZ>
void precond(ok_grid* G, const double* v, TZ* z, cudaStream_t s) {
  if constexpr (std::is_same<TZ, __half>::value) {
    G->pf.apply<TZ>(v, z, s);                     // float16 Z: float32 preconditioner
  } else {
    if (G->o.precision != OK_FP64) G->pf.apply<TZ>(v, z, s);
    else G->pd.apply<TZ>(v, z, s);
  }
}

template <typename TZ>
void arnoldi(ok_grid* G, TZ* Z, int j, cudaStream_t s) {
  const long long N = 2 * G->g0.nv;
  const double* vj = G->V + (long long)j * N;
  double* w = G->V + (long long)(j + 1) * N;
  TZ* zj = Z + (long long)j * N;
  Profiler& pr = G->prof;
  pr.begin(PT_PRECOND, s);
  precond<TZ>(G, vj, zj, s);
  pr.end(PT_PRECOND, s);
  pr.begin(PT_APPLYJ, s);
  launch_apply_j<TZ>(G->dim, G->g0, G->refWM, G->refWK, G->jc, G->coef, zj, w, nullptr, s);
  pr.end(PT_APPLYJ, s);
  pr.begin(PT_CGS2, s);
  if (G->o.reorth == 1) {           // CGS2: always two passes (the default)
    launch_multidot(G->V, N, j + 1, w, N, G->rs, ks_h1_ptr(G->ks), s);
    launch_update_multidot(G->V, N, j + 1, ks_h1_ptr(G->ks), w, N, G->rs, ks_h2_ptr(G->ks), s);
    launch_update_norm_givens(G->V, N, j + 1, w, N, G->rs, G->ks, j, s);
  } else if (G->o.reorth == 2) {    // one classical pass
    launch_multidot(G->V, N, j + 1, w, N, G->rs, ks_h1_ptr(G->ks), s);
    launch_update_norm_check(G->V, N, j + 1, w, N, G->rs, G->ks, j, s, true);
  } else {                          // second pass only when the first cancelled too much
    const int* skip = ks_skip2_ptr(G->ks);
    launch_multidot(G->V, N, j + 1, w, N, G->rs, ks_h1_ptr(G->ks), s, nullptr, ks_nw0_ptr(G->ks));
    launch_update_norm_check(G->V, N, j + 1, w, N, G->rs, G->ks, j, s);
    launch_multidot(G->V, N, j + 1, w, N, G->rs, ks_h2_ptr(G->ks), s, skip);
    launch_update_norm_givens(G->V, N, j + 1, w, N, G->rs, G->ks, j, s, skip);
  }
  launch_scale_by(w, N, ks_eta_ptr(G->ks) + 1, s);   // inv_eta follows eta
  pr.end(PT_CGS2, s);
}

// Arnoldi steps launched per host check when conditional graphs are used
#ifndef OK_COND_BATCH
#define OK_COND_BATCH 4
#endif
static constexpr int COND_BATCH = OK_COND_BATCH;

// Graph of Arnoldi step j behind a device-side condition: a one-thread kernel
// sets the IF node's condition from the cycle's continue flag (the previous
// step's stop test), and the captured step runs only while it is set.  The
// host can then launch several steps and check once.  Returns false (and
// leaves no error) when the device or the captured step cannot be built this
// way; the caller keeps the per-step path.
template <typename TZ>
bool build_cond_graph(ok_grid* G, TZ* Z, int j) {
  cudaStream_t s = G->s;
  for (int attempt = 0; attempt < 2; ++attempt) {
    const bool pdl_saved = g_pdl;
    if (attempt == 1) g_pdl = false;               // programmatic edges inside the body may be refused
    cudaGraph_t gr = nullptr;
    cudaGraphExec_t ex = nullptr;
    cudaGraphConditionalHandle h = 0;
    cudaGraphNode_t kn = nullptr, cn = nullptr;
    bool ok = cudaGraphCreate(&gr, 0) == cudaSuccess;
    ok = ok && cudaGraphConditionalHandleCreate(&h, gr, 0, cudaGraphCondAssignDefault) == cudaSuccess;
    if (ok) {
      KrylovState* ksp = G->ks;
      void* args[] = {&h, &ksp};
      cudaKernelNodeParams kp = {};
      kp.func = cond_set_kernel();
      kp.gridDim = dim3(1, 1, 1);
      kp.blockDim = dim3(1, 1, 1);
      kp.kernelParams = args;
      ok = cudaGraphAddKernelNode(&kn, gr, nullptr, 0, &kp) == cudaSuccess;
    }
    cudaGraph_t body = nullptr;
    if (ok) {
      cudaGraphNodeParams cp = {};
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = h;
      cp.conditional.type = cudaGraphCondTypeIf;
      cp.conditional.size = 1;
      ok = cudaGraphAddNode(&cn, gr, &kn, nullptr, 1, &cp) == cudaSuccess;
      if (ok) body = cp.conditional.phGraph_out[0];
    }
    const long long c0 = g_launch_count.load();
    if (ok) {
      ok = cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
           cudaSuccess;
      if (ok) {
        G->prof.reset_step();
        arnoldi<TZ>(G, Z, j, s);
        cudaGraph_t out = nullptr;
        ok = cudaStreamEndCapture(s, &out) == cudaSuccess;
      }
    }
    const long long c1 = g_launch_count.load();
    g_launch_count.fetch_sub(c1 - c0);              // counted when a body runs
    if (ok) ok = cudaGraphInstantiate(&ex, gr, 0) == cudaSuccess;
    if (gr) cudaGraphDestroy(gr);
    g_pdl = pdl_saved;
    if (ok) {
      G->cgraphs[j] = ex;
      G->cgraph_kernels[j] = c1 - c0;
      return true;
    }
    cudaGetLastError();
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
      cudaGraph_t dead = nullptr;
      cudaStreamEndCapture(s, &dead);
      if (dead) cudaGraphDestroy(dead);
    }
    cudaGetLastError();
    if (ex) cudaGraphExecDestroy(ex);
  }
  return false;
}

// Right-preconditioned restarted FGMRES for J x = f (all device pointers).
template <typename TZ>
void fgmres(ok_grid* G, TZ* Z, const double* f, double* x, int& its, double& rel) {
  cudaStream_t s = G->s;
  const long long N = 2 * G->g0.nv;
  const int m = G->o.restart;
  const double rtol = G->o.gmres_rtol;
  its = 0;
  launch_norm(f, N, G->rs, G->dsc, s);
  CKL();
  const double fnorm = read_scalar(G, G->dsc);
  CK(cudaMemsetAsync(x, 0, N * sizeof(double), s));
  if (!std::isfinite(fnorm)) fail(OK_ERR_NONFINITE, "non-finite right-hand side");
  if (fnorm == 0.0) {
    rel = 0.0;
    return;
  }
  CK(cudaMemcpyAsync(G->rv, f, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  double beta = fnorm;
  CK(cudaMemcpyAsync(G->dsc + 1, G->dsc, sizeof(double), cudaMemcpyDeviceToDevice, s));
  const bool graphs = G->o.use_graphs != 0;
  while (beta > rtol * fnorm && its < G->o.max_gmres) {
    launch_cycle_start(G->ks, G->dsc + 1, rtol * fnorm, s);
    launch_axpby<double, double>(N, 1.0, G->rv, 0.0, G->V, s);
    launch_scale_by(G->V, N, ks_beta_ptr(G->ks) + 1, s);    // inv_beta follows beta
    CKL();
    int jused = 0;
    const int jmax = std::min(m, G->o.max_gmres - its);
    bool stop = false;
    while (!stop && jused < jmax) {
      if (graphs && !G->prof.on && G->cond_ok) {
        // up to COND_BATCH steps behind device-side conditions, one host check
        const int nb = std::min(COND_BATCH, jmax - jused);
        int launched = 0;
        for (int b = 0; b < nb; ++b) {
          const int jj = jused + b;
          if (!G->cgraphs[jj] && !build_cond_graph<TZ>(G, Z, jj)) break;
          CK(cudaGraphLaunch(G->cgraphs[jj], s));
          ++launched;
        }
        if (launched > 0) {
          CK(cudaMemcpyAsync(G->hpin, ks_eta_ptr(G->ks), 5 * sizeof(double), cudaMemcpyDeviceToHost, s));
          CK(cudaStreamSynchronize(s));
          const double est = G->hpin[2], go = G->hpin[3];
          const int taken = (int)G->hpin[4];
          long long k = launched;                       // the condition kernels
          for (int jj = jused; jj < taken; ++jj) k += G->cgraph_kernels[jj];
          g_launch_count.fetch_add(k);
          its += taken - jused;
          jused = taken;
          if (!std::isfinite(est)) fail(OK_ERR_NONFINITE, "non-finite value in FGMRES");
          stop = go == 0.0;
          continue;
        }
        G->cond_ok = false;                             // per-step graphs from here on
      }
      const int j = jused;
      TagSet tags;
      if (graphs && !G->graphs[j]) {
        // A capture can be invalidated by another host thread's context-wide
        // work (e.g. loading a module on first use); the step then runs
        // uncaptured and the capture is tried again at the next cycle.
        cudaGraph_t gr = nullptr;
        G->prof.reset_step();
        const long long c0 = g_launch_count.load();
        cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
          arnoldi<TZ>(G, Z, j, s);
          e = cudaStreamEndCapture(s, &gr);
        }
        const long long c1 = g_launch_count.load();
        g_launch_count.fetch_sub(c1 - c0);            // counted when the graph runs
        if (e == cudaSuccess && gr) e = cudaGraphInstantiate(&G->graphs[j], gr, 0);
        if (gr) cudaGraphDestroy(gr);
        if (e == cudaSuccess && G->graphs[j]) {
          G->graph_kernels[j] = c1 - c0;
          G->graph_tags[j] = G->prof.ended;
        } else {
          cudaGetLastError();
          cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
          if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
            cudaGraph_t dead = nullptr;
            cudaStreamEndCapture(s, &dead);
            if (dead) cudaGraphDestroy(dead);
          }
          cudaGetLastError();
          if (G->graphs[j]) cudaGraphExecDestroy(G->graphs[j]);
          G->graphs[j] = nullptr;
        }
      }
      if (graphs && G->graphs[j]) {
        CK(cudaGraphLaunch(G->graphs[j], s));
        g_launch_count.fetch_add(G->graph_kernels[j]);
        tags = G->graph_tags[j];
      } else {
        G->prof.reset_step();
        arnoldi<TZ>(G, Z, j, s);
        CKL();
        tags = G->prof.ended;
      }
      ++its;
      jused = j + 1;
      CK(cudaMemcpyAsync(G->hpin, ks_eta_ptr(G->ks), 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (G->prof.on) G->prof.collect(tags);
      const double eta = G->hpin[0], est = G->hpin[2];
      if (!std::isfinite(est)) fail(OK_ERR_NONFINITE, "non-finite value in FGMRES");
      stop = est <= rtol * fnorm || eta == 0.0;
    }
    launch_lsq(G->ks, jused, s);
    launch_multi_axpy<TZ>(Z, N, jused, G->ks, x, N, s);
    JCoefs jc = G->jc;
    jc.alpha = -1.0;
    jc.beta = 1.0;
    launch_apply_j<double>(G->dim, G->g0, G->refWM, G->refWK, jc, G->coef, x, G->rv, f, s);   // r = f - J x
    launch_norm(G->rv, N, G->rs, G->dsc + 1, s);
    CKL();
    beta = read_scalar(G, G->dsc + 1);
    if (!std::isfinite(beta)) fail(OK_ERR_NONFINITE, "non-finite residual in FGMRES");
  }
  rel = beta / fnorm;
}

void linear_solve(ok_grid* G, const double* f, double* x, int& its, double& rel) {
  if (G->o.precision == OK_MIXED) fgmres<float>(G, G->Zf, f, x, its, rel);
  else if (G->o.precision == OK_MIXED_HALF) fgmres<__half>(G, G->Zh, f, x, its, rel);
  else fgmres<double>(G, G->Zd, f, x, its, rel);
}

// f = -F(u_k, w_k), returns ||F||_2
double residual(ok_grid* G, const double* un, const double* wn, const double* uk, const double* wk, double* f) {
  launch_residual(G->dim, G->g0, G->refWM, G->refWK, G->rc, un, wn, uk, wk, f, G->s);
  CKL();
  launch_norm(f, 2 * G->g0.nv, G->rs, G->dsc, G->s);
  CKL();
  return read_scalar(G, G->dsc);
}

// one Newton step on the handle's device buffers un, wn, uk, wk
void newton_update(ok_grid* G, ok_step_info& info, double& ms) {
  auto t0 = std::chrono::steady_clock::now();
  assemble_c(G, G->uk);
  int its = 0;
  double rel = 0;
  linear_solve(G, G->f, G->xs, its, rel);
  const long long nv = G->g0.nv;
  launch_axpby<double, double>(nv, 1.0, G->xs, 1.0, G->uk, G->s);
  launch_axpby<double, double>(nv, 1.0, G->xs + nv, 1.0, G->wk, G->s);
  CKL();
  CK(cudaStreamSynchronize(G->s));
  ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  info.gmres_its += its;
  info.last_gmres_its = its;
  info.rel_resid = rel;
  info.newton_its += 1;
  if (rel > G->o.gmres_rtol) fail(OK_ERR_NOT_CONVERGED, "FGMRES did not reach gmres_rtol within max_gmres");
}

void copy_out(ok_grid* G, double* dst, const double* src, long long count) {
  CK(cudaMemcpyAsync(dst, src, count * sizeof(double), cudaMemcpyDefault, G->s));
}

// x^T y of two device vectors (deterministic two-stage reduction), on the host
double dot(ok_grid* G, const double* x, const double* y, long long n) {
  launch_multidot(x, n, 1, y, n, G->rs, G->dsc + 2, G->s);
  CKL();
  return read_scalar(G, G->dsc + 2);
}

void energy_setup(ok_grid* G) {
  if (G->ew) return;
  std::unique_ptr<EnergyWork> E(new EnergyWork());
  const int dim = G->dim;
  const int NOFF = dim == 2 ? Topo<2>::NOFF : Topo<3>::NOFF;
  const int NCLASS = dim == 2 ? Topo<2>::NCLASS : Topo<3>::NCLASS;
  std::vector<double> refM(NCLASS * NOFF), refK(NCLASS * NOFF);
  reference_tables(dim, refM.data(), refK.data());
  build_prec<double>(G, E->mg, level_sizes(G->n, G->o.coarse_max), refM, refK, 1.0);   // M + K
  E->mg.n_V = 2;
  E->mg.prof = nullptr;
  const long long nv = G->g0.nv;
  Arena& A = G->arena;
  for (double** v : {&E->ones, &E->lm, &E->f, &E->b, &E->x, &E->r, &E->z, &E->p, &E->q}) *v = A.alloc<double>(nv);
  E->e = A.alloc<double>(2 * nv);
  std::vector<double> one(nv, 1.0);
  CK(cudaMemcpy(E->ones, one.data(), nv * sizeof(double), cudaMemcpyHostToDevice));
  launch_op_apply<double, double, double>(dim, G->g0, G->WM0d, false, E->ones, E->lm, 1.0, (const double*)nullptr,
                                          0.0, G->s);            // 1^T M, the lumped masses
  CKL();
  CK(cudaStreamSynchronize(G->s));
  G->ew = E.release();
}

// The three terms of the Ohta--Kawasaki energy (Sec. 1) of the device vector u.
void energy(ok_grid* G, const double* u, double out[3]) {
  energy_setup(G);
  EnergyWork& E = *G->ew;
  const long long nv = G->g0.nv;
  const int dim = G->dim;
  cudaStream_t s = G->s;
  launch_energy_local(dim, G->g0, G->refWK, G->rc, u, E.e, s);
  CKL();
  out[0] = dot(G, E.ones, E.e, nv);
  out[1] = dot(G, E.ones, E.e + nv, nv);
  // f = u - (1^T M u) / |Omega|, mean-free; b = M f
  const double mean = dot(G, E.lm, u, nv) / dot(G, E.lm, E.ones, nv);
  CK(cudaMemcpyAsync(E.f, u, nv * sizeof(double), cudaMemcpyDeviceToDevice, s));
  launch_axpby<double, double>(nv, -mean, E.ones, 1.0, E.f, s);
  launch_op_apply<double, double, double>(dim, G->g0, G->WM0d, false, E.f, E.b, 1.0, (const double*)nullptr, 0.0,
                                          s);
  CKL();
  // 1^T b = 1^T M f = 0 up to rounding; remove that rounding (the component of
  // b along the null vector 1 of K), else CG stalls at its size when f is
  // itself at rounding level (a constant u)
  const double bsum = dot(G, E.ones, E.b, nv);
  launch_axpby<double, double>(nv, -bsum / (double)nv, E.ones, 1.0, E.b, s);
  CKL();
  // conjugate gradients for K x = b (consistent: 1^T b = 0), preconditioned by
  // two V-cycles for M + K (symmetric: the same Chebyshev polynomial before and
  // after the coarse correction); stop at ||r|| <= 1e-12 ||b||
  const double bn = std::sqrt(dot(G, E.b, E.b, nv));
  CK(cudaMemsetAsync(E.x, 0, nv * sizeof(double), s));
  double xb = 0.0;
  E.last_its = 0;
  if (bn > 0.0) {
    CK(cudaMemcpyAsync(E.r, E.b, nv * sizeof(double), cudaMemcpyDeviceToDevice, s));
    E.mg.solve_mg(E.r, E.z, s);
    CK(cudaMemcpyAsync(E.p, E.z, nv * sizeof(double), cudaMemcpyDeviceToDevice, s));
    double rz = dot(G, E.r, E.z, nv);
    const double hk = G->rc.hk;
    for (int it = 0; it < 500; ++it) {
      launch_op_apply<double, double, double>(dim, G->g0, G->refWK, true, E.p, E.q, hk, (const double*)nullptr,
                                              0.0, s);
      CKL();
      const double al = rz / dot(G, E.p, E.q, nv);
      launch_axpby<double, double>(nv, al, E.p, 1.0, E.x, s);
      launch_axpby<double, double>(nv, -al, E.q, 1.0, E.r, s);
      E.last_its = it + 1;
      const double rn = std::sqrt(dot(G, E.r, E.r, nv));
      if (!std::isfinite(rn)) fail(OK_ERR_NONFINITE, "non-finite residual in the energy's Neumann solve");
      if (rn <= 1e-12 * bn) break;
      E.mg.solve_mg(E.r, E.z, s);
      const double rz1 = dot(G, E.r, E.z, nv);
      launch_axpby<double, double>(nv, 1.0, E.z, rz1 / rz, E.p, s);
      CKL();
      rz = rz1;
    }
    xb = dot(G, E.b, E.x, nv);
  }
  out[2] = 0.5 * G->p.sigma * xb;
}

// ---------------------------------------------------------------------------
// Cohorts (ok_solve_batch): problems with the same grid, options and
// multigrid structure advance in lockstep, and every kernel of an Arnoldi step
// (the preconditioner's stencil and multigrid kernels, J z and the CGS2
// orthogonalisation) runs as one launch over all of them.  Each problem's
// arithmetic is the one it gets alone: same kernel bodies, same reduction
// shapes, same stop decisions (taken per problem), so the results are bitwise
// those of ok_timestep.
// ---------------------------------------------------------------------------
template <typename T>
bool same_structure(const Prec<T>& a, const Prec<T>& b) {
  if (a.lv.size() != b.lv.size() || a.tiled != b.tiled || a.fused != b.fused || a.Lc != b.Lc ||
      a.low != b.low || a.cheb_coarse != b.cheb_coarse || a.plane3 != b.plane3 || a.pshape != b.pshape ||
      (a.gemv_inv == nullptr) != (b.gemv_inv == nullptr) || a.gemv_ldA != b.gemv_ldA || a.k_R != b.k_R ||
      a.n_V != b.n_V || a.q_A != b.q_A || a.nu_pre != b.nu_pre || a.nu_post != b.nu_post || a.csmem != b.csmem)
    return false;
  if (a.tiled)
    for (size_t l = 0; l + 1 < a.lv.size(); ++l)
      if (a.ts[l].tile != b.ts[l].tile) return false;
  return true;
}

// may handles a and b share launches?
bool cohort_compatible(const ok_grid* a, const ok_grid* b) {
  const ok_opts &x = a->o, &y = b->o;
  if (a->dim != b->dim || a->n != b->n || a->device != b->device || x.precision != y.precision ||
      x.restart != y.restart || x.reorth != 1 || y.reorth != 1 || x.use_pdl != y.use_pdl ||
      x.max_gmres != y.max_gmres || x.fuse_coarse == 2 || y.fuse_coarse == 2)
    return false;
  return x.precision == OK_FP64 ? same_structure(a->pd, b->pd) : same_structure(a->pf, b->pf);
}

template <typename T>
struct CohortPrec {
  std::vector<Prec<T>*> P;
  int dim = 0;
  int B() const { return (int)P.size(); }
  Prec<T>& p0() { return *P[0]; }

  // ---- 2D register-strip path (Prec::apply_tiled) -------------------------
  template <typename TO>
  void vcycle_t(int l, bool x_zero, T* const* rhs, TO* const* out, T* const* mx, cudaStream_t s) {
    Prec<T>& P0 = p0();
    const int nb = B();
    if (P0.fused && l == P0.Lc) {
      CoarseVItem<T> it[BATCH_MAX];
      for (int i = 0; i < nb; ++i) it[i] = {P[i]->ca_dev, rhs[i], x_zero ? (const T*)nullptr : P[i]->X(l), P[i]->X(l)};
      launch_coarse_vcycle_b<T>(dim, it, nb, P0.csmem, s);
      return;
    }
    if (l + 1 == (int)P0.lv.size()) {
      if (P0.cheb_coarse) {
        for (int i = 0; i < nb; ++i) P[i]->coarse_solve(rhs[i], P[i]->X(l), s);
      } else {
        GemvItem<T> it[BATCH_MAX];
        for (int i = 0; i < nb; ++i)
          it[i] = {P0.gemv_inv ? P[i]->gemv_inv : P[i]->coarse_inv, rhs[i], P[i]->X(l)};
        launch_coarse_solve_b<T>(P0.nc, P0.gemv_ldA, P0.gemv_inv != nullptr, it, nb, s);
      }
      return;
    }
    StripPreItem<T> pre[BATCH_MAX];
    T* nb_rhs[BATCH_MAX];
    for (int i = 0; i < nb; ++i) {
      Prec<T>& Q = *P[i];
      pre[i] = {Q.ts[l], x_zero ? (const T*)nullptr : Q.X(l), rhs[i], Q.Xalt(l), Q.lv[l + 1].b};
      nb_rhs[i] = Q.lv[l + 1].b;
    }
    launch_tile_pre_b<T>(pre, nb, s);
    for (int i = 0; i < nb; ++i) P[i]->cur[l] ^= 1;
    T* none[BATCH_MAX] = {};
    vcycle_t<T>(l + 1, true, nb_rhs, none, none, s);
    StripPostItem<T, TO> post[BATCH_MAX];
    for (int i = 0; i < nb; ++i) {
      Prec<T>& Q = *P[i];
      post[i] = {Q.ts[l], Q.X(l), Q.X(l + 1), rhs[i], Q.Xalt(l), mx[i], out[i], (T)1};
    }
    launch_tile_post_b<T, TO>(post, nb, s);
    for (int i = 0; i < nb; ++i) P[i]->cur[l] ^= 1;
  }
  template <typename TO>
  void mg_solve_t(T* const* rhs, TO* const* out, T* const* mx, cudaStream_t s) {
    for (auto* Q : P) std::fill(Q->cur.begin(), Q->cur.end(), 0);
    TO* no_out[BATCH_MAX] = {};
    T* no_mx[BATCH_MAX] = {};
    for (int c = 0; c < p0().n_V; ++c) {
      const bool last = c + 1 == p0().n_V;
      vcycle_t<TO>(0, c == 0, rhs, last ? out : no_out, last ? mx : no_mx, s);
    }
  }

  // ---- per-level steps (3D, or untiled): Prec::cheb with shared launches ---
  // (the output scale is per member: the mass solve divides by each member's
  // own 1 + dt theta sigma)
  template <typename TB, typename TO>
  void cheb(int l, bool mass, const TB* const* b, bool x_zero, int steps, TO* const* out, const T* oscale,
            bool want_r, cudaStream_t s, bool inited = false, const T** defer_last = nullptr) {
    Prec<T>& P0 = p0();
    const int nb = B();
    const Geom& g = P0.lv[l].g;
    const double th = mass ? P0.thM : P0.thS;
    const std::vector<double>& c1 = mass ? P0.cM1 : P0.cS1;
    const std::vector<double>& c2 = mass ? P0.cM2 : P0.cS2;
    auto W = [&](int i) { return mass ? P[i]->WM : P[i]->lv[l].WS; };
    auto dinv = [&](int i) { return mass ? P[i]->dinvM : P[i]->lv[l].dinvS; };
    auto X = [&](int i) { return mass ? P[i]->cx : P[i]->lv[l].x; };
    auto R = [&](int i) { return mass ? P[i]->cr : P[i]->lv[l].r; };
    auto D0 = [&](int i) { return mass ? P[i]->cd0 : P[i]->lv[l].d0; };
    auto D1 = [&](int i) { return mass ? P[i]->cd1 : P[i]->lv[l].d1; };
    const int shape = P0.plane_shape(g);
    if (x_zero && inited) {
      // r and d0 written by the restriction launch
    } else if (x_zero) {
      ChebInitItem<T, TB> it[BATCH_MAX];
      for (int i = 0; i < nb; ++i) it[i] = {dinv(i), b[i], (T)1, R(i), D0(i), (T)(1.0 / th)};
      launch_cheb_init_b<T, TB>(dim, g, it, nb, s);
    } else if (P0.on_planes(g)) {
      PlaneArgs<T, T, T> it[BATCH_MAX];
      for (int i = 0; i < nb; ++i) {
        it[i] = {};
        it[i].g = g, it[i].W = W(i), it[i].dinv = dinv(i), it[i].s = X(i), it[i].r = R(i), it[i].d = D0(i);
        it[i].b = (const T*)b[i], it[i].inv_th = (T)(1.0 / th);
      }
      launch_plane3_b<T, T, T>(PM_RESID, it, nb, shape, s);
    } else {
      for (int i = 0; i < nb; ++i)
        launch_resid_init<T>(dim, g, W(i), dinv(i), (const T*)b[i], X(i), R(i), D0(i), (T)(1.0 / th), s);
    }
    int cur = 0;
    for (int k = 0; k + 1 < steps; ++k) {
      const bool first = x_zero && k == 0;
      if (P0.on_planes(g)) {
        PlaneArgs<T, T, T> it[BATCH_MAX];
        for (int i = 0; i < nb; ++i) {
          T* d[2] = {D0(i), D1(i)};
          it[i] = {};
          it[i].g = g, it[i].W = W(i), it[i].dinv = dinv(i), it[i].s = d[cur], it[i].x = X(i), it[i].r = R(i);
          it[i].d = d[1 - cur], it[i].c1 = (T)c1[k], it[i].c2 = (T)c2[k], it[i].first = first ? 1 : 0;
        }
        launch_plane3_b<T, T, T>(PM_STEP, it, nb, shape, s);
      } else {
        for (int i = 0; i < nb; ++i) {
          T* d[2] = {D0(i), D1(i)};
          launch_cheb_step<T>(dim, g, W(i), dinv(i), X(i), R(i), d[cur], d[1 - cur], (T)c1[k], (T)c2[k], first, s);
        }
      }
      cur ^= 1;
    }
    const bool first = x_zero && steps == 1;
    bool no_out = true;
    for (int i = 0; i < nb; ++i) no_out = no_out && out[i] == nullptr;
    if (defer_last && !want_r && no_out && !first) {
      for (int i = 0; i < nb; ++i) {
        T* d[2] = {D0(i), D1(i)};
        defer_last[i] = d[cur];
      }
      return;
    }
    if (P0.on_planes(g) && want_r) {
      PlaneArgs<T, T, T> it[BATCH_MAX];
      for (int i = 0; i < nb; ++i) {
        T* d[2] = {D0(i), D1(i)};
        it[i] = {};
        it[i].g = g, it[i].W = W(i), it[i].s = d[cur], it[i].x = X(i), it[i].r = R(i), it[i].first = first ? 1 : 0;
        it[i].out = (T*)out[i], it[i].oscale = oscale[i];
      }
      launch_plane3_b<T, T, T>(PM_LAST, it, nb, shape, s);
    } else {
      ChebLastItem<T, TO> it[BATCH_MAX];
      for (int i = 0; i < nb; ++i) {
        T* d[2] = {D0(i), D1(i)};
        it[i] = {W(i), X(i), want_r ? R(i) : (T*)nullptr, d[cur], first ? 1 : 0, out[i], oscale[i]};
      }
      launch_cheb_last_b<T, TO>(dim, g, it, nb, s);
    }
  }

  template <typename TO>
  void vcycle(int l, bool x_zero, TO* const* out, cudaStream_t s, bool inited = false, const T** defer = nullptr) {
    Prec<T>& P0 = p0();
    const int nb = B();
    const bool coarsest = l + 1 == (int)P0.lv.size();
    if ((P0.fused && l == P0.Lc) || coarsest) {
      if (P0.fused && l == P0.Lc) {
        CoarseVItem<T> it[BATCH_MAX];
        for (int i = 0; i < nb; ++i) {
          Level<T>& L = P[i]->lv[l];
          it[i] = {P[i]->ca_dev, L.b, x_zero ? (const T*)nullptr : L.x, L.x};
        }
        launch_coarse_vcycle_b<T>(dim, it, nb, P0.csmem, s);
      } else if (P0.cheb_coarse) {
        for (int i = 0; i < nb; ++i) P[i]->coarse_solve(P[i]->lv[l].b, P[i]->lv[l].x, s);
      } else {
        GemvItem<T> it[BATCH_MAX];
        for (int i = 0; i < nb; ++i)
          it[i] = {P0.gemv_inv ? P[i]->gemv_inv : P[i]->coarse_inv, P[i]->lv[l].b, P[i]->lv[l].x};
        launch_coarse_solve_b<T>(P0.nc, P0.gemv_ldA, P0.gemv_inv != nullptr, it, nb, s);
      }
      for (int i = 0; i < nb; ++i)
        if (out[i]) launch_axpby<T, TO>(P[i]->lv[l].g.nv, 1.0, P[i]->lv[l].x, 0.0, out[i], s);
      return;
    }
    T* none[BATCH_MAX] = {};
    T* bl[BATCH_MAX];
    T ones[BATCH_MAX];
    for (int i = 0; i < nb; ++i) bl[i] = P[i]->lv[l].b, ones[i] = (T)1;
    cheb<T, T>(l, false, bl, x_zero, P0.nu_pre, none, ones, true, s, inited);
    const Geom& gf = P0.lv[l].g;
    const Geom& gc = P0.lv[l + 1].g;
    const bool c_smooths = !(P0.fused && l + 1 == P0.Lc) && l + 2 < (int)P0.lv.size();   // as Prec::vcycle
    TransferItem<T> tr[BATCH_MAX];
    for (int i = 0; i < nb; ++i) {
      Level<T>& C = P[i]->lv[l + 1];
      tr[i] = {P[i]->lv[l].r, C.b};
      if (c_smooths) tr[i].dinv = C.dinvS, tr[i].r = C.r, tr[i].d = C.d0, tr[i].inv_th = (T)(1.0 / P0.thS);
    }
    launch_restrict_b<T>(dim, gf, gc, tr, nb, s);
    const T* dc[BATCH_MAX] = {};
    vcycle<T>(l + 1, true, none, s, c_smooths, c_smooths ? dc : nullptr);
    for (int i = 0; i < nb; ++i) {
      tr[i] = {P[i]->lv[l].x, P[i]->lv[l + 1].x};
      tr[i].dc = dc[i];
    }
    launch_prolong_add_b<T>(dim, gf, gc, tr, nb, s);
    cheb<T, TO>(l, false, bl, false, P0.nu_post, out, ones, false, s, false, defer);
  }
  template <typename TO>
  void mg_solve(TO* const* out, cudaStream_t s) {
    TO* none[BATCH_MAX] = {};
    for (int c = 0; c < p0().n_V; ++c) vcycle<TO>(0, c == 0, c + 1 == p0().n_V ? out : none, s);
  }

  // z_i = P_i^{-1} v_i for every member
  template <typename TZ>
  void apply(const double* const* v, TZ* const* z, cudaStream_t s) {
    Prec<T>& P0 = p0();
    const int nb = B();
    const long long nv = P0.lv[0].g.nv;
    if (P0.tiled) {
      AmassItem<T, TZ> am[BATCH_MAX];
      T *b0[BATCH_MAX], *b2[BATCH_MAX];
      TZ* z2[BATCH_MAX];
      T* none[BATCH_MAX] = {};
      TZ* nonez[BATCH_MAX] = {};
      for (int i = 0; i < nb; ++i) {
        am[i] = {P[i]->tm, v[i], z[i], P[i]->lv[0].b};
        b0[i] = P[i]->lv[0].b;
        b2[i] = P[i]->b2;
        z2[i] = z[i] + nv;
      }
      launch_tile_amass_b<T, TZ>(am, nb, s);
      mg_solve_t<T>(b0, none, b2, s);                                 // b2 = M S_hat^{-1} t
      (void)nonez;
      mg_solve_t<TZ>(b2, z2, none, s);                                // z2 = S_hat^{-1} b2
      return;
    }
    if (P0.k_R != 1) {                                                // two Richardson steps: per problem
      for (int i = 0; i < nb; ++i) P[i]->template apply<TZ>(v[i], z[i], s);
      return;
    }
    const Geom& g = P0.lv[0].g;
    T ia[BATCH_MAX];
    for (int i = 0; i < nb; ++i) ia[i] = (T)P[i]->inv_a11;
    cheb<double, TZ>(0, true, v, true, P0.q_A, z, ia, false, s);                    // z1 = A~^{-1} r1
    CStepItem<T, double> cs[BATCH_MAX];
    for (int i = 0; i < nb; ++i) cs[i] = {P[i]->coef, v[i] + nv, (T)1, P[i]->cx, (T)P[i]->inv_a11, P[i]->lv[0].b};
    launch_cstep_b<T, double>(dim, g, cs, nb, s);                     // t = r2 - C z1
    T* none[BATCH_MAX] = {};
    mg_solve<T>(none, s);                                             // S_hat^{-1} t
    if (P0.on_planes(g)) {                                            // M .
      PlaneArgs<T, T, T> it[BATCH_MAX];
      for (int i = 0; i < nb; ++i) {
        it[i] = {};
        it[i].g = g, it[i].W = P[i]->WM, it[i].s = P[i]->lv[0].x, it[i].out = P[i]->lv[0].b, it[i].alpha = (T)1;
      }
      launch_plane3_b<T, T, T>(PM_OP, it, nb, P0.plane_shape(g), s);
    } else {
      for (int i = 0; i < nb; ++i) P[i]->op(g, P[i]->WM, false, P[i]->lv[0].x, P[i]->lv[0].b, (T)1, s);
    }
    TZ* z2[BATCH_MAX];
    for (int i = 0; i < nb; ++i) z2[i] = z[i] + nv;
    mg_solve<TZ>(z2, s);                                              // S_hat^{-1} .
  }
};

// Arnoldi step j of every member: z_j = P^{-1} v_j, w = J z_j, CGS2 of w
template <typename TZ>
void arnoldi_b(const std::vector<ok_grid*>& Gs, const std::vector<TZ*>& Zs, int j, cudaStream_t s) {
  const int nb = (int)Gs.size();
  ok_grid* G0 = Gs[0];
  const long long N = 2 * G0->g0.nv;
  const double* v[BATCH_MAX];
  TZ* z[BATCH_MAX];
  for (int i = 0; i < nb; ++i) {
    v[i] = Gs[i]->V + (long long)j * N;
    z[i] = Zs[i] + (long long)j * N;
  }
  if constexpr (std::is_same<TZ, double>::value) {        // float64 Z: the float64 preconditioner
    CohortPrec<double> cp;
    cp.dim = G0->dim;
    for (auto* G : Gs) cp.P.push_back(&G->pd);
    cp.apply<TZ>(v, z, s);
  } else {                                                 // float32 / float16 Z: the float32 one
    CohortPrec<float> cp;
    cp.dim = G0->dim;
    for (auto* G : Gs) cp.P.push_back(&G->pf);
    cp.apply<TZ>(v, z, s);
  }
  ApplyJItem<TZ> aj[BATCH_MAX];
  KrylovItem kr[BATCH_MAX];
  for (int i = 0; i < nb; ++i) {
    ok_grid* G = Gs[i];
    double* w = G->V + (long long)(j + 1) * N;
    aj[i] = {G->jc, G->coef, z[i], w};
    kr[i] = {G->V, N, w, N, G->rs.partials, G->rs.counter, G->ks, 0};
  }
  launch_apply_j_b<TZ>(G0->dim, G0->g0, G0->refWM, G0->refWK, aj, nb, s);
  launch_cgs2_batch(kr, nb, j + 1, j, s);
  CKL();
}

// Lockstep restarted FGMRES for the members' systems J_i x_i = f_i (the
// members' own f and xs buffers); per-member iteration counts and relative
// residuals; a member that fails gets its status and leaves the cohort.
template <typename TZ>
void fgmres_b(const std::vector<ok_grid*>& Gs, const std::vector<TZ*>& Zs, std::vector<int>& its,
              std::vector<double>& rel, std::vector<int>& status, cudaStream_t s) {
  const int nb = (int)Gs.size();
  ok_grid* G0 = Gs[0];
  const long long N = 2 * G0->g0.nv;
  const int m = G0->o.restart;
  const double rtol = G0->o.gmres_rtol;
  std::vector<double> fnorm(nb, 0.0), beta(nb, 0.0);
  std::vector<int> active;
  for (int i = 0; i < nb; ++i) {
    ok_grid* G = Gs[i];
    its[i] = 0;
    rel[i] = 0.0;
    launch_norm(G->f, N, G->rs, G->dsc, s);
    CKL();
    CK(cudaMemcpyAsync(G->hpin, G->dsc, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaMemsetAsync(G->xs, 0, N * sizeof(double), s));
  }
  CK(cudaStreamSynchronize(s));
  for (int i = 0; i < nb; ++i) {
    ok_grid* G = Gs[i];
    fnorm[i] = G->hpin[0];
    if (!std::isfinite(fnorm[i])) {
      status[i] = OK_ERR_NONFINITE;
      continue;
    }
    if (fnorm[i] == 0.0) continue;
    CK(cudaMemcpyAsync(G->rv, G->f, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(G->dsc + 1, G->dsc, sizeof(double), cudaMemcpyDeviceToDevice, s));
    beta[i] = fnorm[i];
    if (beta[i] > rtol * fnorm[i]) active.push_back(i);
  }
  while (!active.empty()) {
    std::vector<int> jmax(nb, 0), jused(nb, 0);
    for (int i : active) {
      ok_grid* G = Gs[i];
      launch_cycle_start(G->ks, G->dsc + 1, rtol * fnorm[i], s);
      launch_axpby<double, double>(N, 1.0, G->rv, 0.0, G->V, s);
      launch_scale_by(G->V, N, ks_beta_ptr(G->ks) + 1, s);
      CKL();
      jmax[i] = std::min(m, G->o.max_gmres - its[i]);
    }
    std::vector<int> cyc = active;
    for (int j = 0; !cyc.empty(); ++j) {
      std::vector<ok_grid*> g;
      std::vector<TZ*> z;
      for (int i : cyc) g.push_back(Gs[i]), z.push_back(Zs[i]);
      arnoldi_b<TZ>(g, z, j, s);
      for (int i : cyc)
        CK(cudaMemcpyAsync(Gs[i]->hpin, ks_eta_ptr(Gs[i]->ks), 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      std::vector<int> next;
      for (int i : cyc) {
        its[i] += 1;
        jused[i] = j + 1;
        const double est = Gs[i]->hpin[2], go = Gs[i]->hpin[3];
        if (!std::isfinite(est)) {
          status[i] = OK_ERR_NONFINITE;
          continue;
        }
        if (go != 0.0 && j + 1 < jmax[i]) next.push_back(i);
      }
      cyc.swap(next);
    }
    std::vector<int> still;
    for (int i : active) {
      if (status[i] != OK_SUCCESS) continue;
      ok_grid* G = Gs[i];
      launch_lsq(G->ks, jused[i], s);
      launch_multi_axpy<TZ>(Zs[i], N, jused[i], G->ks, G->xs, N, s);
      JCoefs jc = G->jc;
      jc.alpha = -1.0;
      jc.beta = 1.0;
      launch_apply_j<double>(G->dim, G->g0, G->refWM, G->refWK, jc, G->coef, G->xs, G->rv, G->f, s);
      launch_norm(G->rv, N, G->rs, G->dsc + 1, s);
      CKL();
      CK(cudaMemcpyAsync(G->hpin + 4, G->dsc + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
    }
    CK(cudaStreamSynchronize(s));
    for (int i : active) {
      if (status[i] != OK_SUCCESS) continue;
      beta[i] = Gs[i]->hpin[4];
      if (!std::isfinite(beta[i])) {
        status[i] = OK_ERR_NONFINITE;
        continue;
      }
      if (beta[i] > rtol * fnorm[i] && its[i] < Gs[i]->o.max_gmres) still.push_back(i);
    }
    active.swap(still);
  }
  for (int i = 0; i < nb; ++i)
    if (fnorm[i] > 0.0 && std::isfinite(fnorm[i])) rel[i] = beta[i] / fnorm[i];
}

// Every member's stream is the cohort's stream while the cohort runs (the
// per-member helpers enqueue on G->s), restored afterwards.
struct CohortStreams {
  std::vector<ok_grid*> Gs;
  std::vector<cudaStream_t> saved;
  CohortStreams(const std::vector<ok_grid*>& g, cudaStream_t s) : Gs(g) {
    for (auto* G : Gs) saved.push_back(G->s), G->s = s;
    g_pdl = Gs[0]->o.use_pdl != 0;
  }
  ~CohortStreams() {
    for (size_t i = 0; i < Gs.size(); ++i) Gs[i]->s = saved[i];
  }
};

// One theta-method timestep for every member (state in/out through u[i],
// w[i]), Newton in lockstep: the members that still need a Newton step share
// the linear solve's launches.
void timestep_b(const std::vector<ok_grid*>& Gs, double* const* u, double* const* w, std::vector<ok_step_info>& info,
                std::vector<int>& status, cudaStream_t s) {
  const int nb = (int)Gs.size();
  const long long nv = Gs[0]->g0.nv;
  std::vector<double> fn(nb, 0.0), r0(nb, 0.0);
  std::vector<int> extra(nb, 0), done(nb, 0), ok(nb, 0);
  for (int i = 0; i < nb; ++i) {
    ok_grid* G = Gs[i];
    std::memset(&info[i], 0, sizeof(ok_step_info));
    CK(cudaMemcpyAsync(G->un, u[i], nv * sizeof(double), cudaMemcpyDefault, s));
    CK(cudaMemcpyAsync(G->wn, w[i], nv * sizeof(double), cudaMemcpyDefault, s));
    CK(cudaMemsetAsync(G->dflag, 0, sizeof(int), s));
    launch_check_finite(G->un, nv, G->dflag, s);
    launch_check_finite(G->wn, nv, G->dflag, s);
    CK(cudaMemcpyAsync(G->uk, G->un, nv * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(G->wk, G->wn, nv * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CKL();
  }
  for (int i = 0; i < nb; ++i) {
    ok_grid* G = Gs[i];
    int flag = 0;
    CK(cudaMemcpyAsync(G->hpin, G->dflag, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    std::memcpy(&flag, G->hpin, sizeof(int));
    if (flag) {
      status[i] = OK_ERR_NONFINITE;
      done[i] = 1;
      continue;
    }
    fn[i] = r0[i] = residual(G, G->un, G->wn, G->uk, G->wk, G->f);
    info[i].newton_resid0 = r0[i];
  }
  std::vector<int> linear_failed(nb, 0);
  auto t0 = std::chrono::steady_clock::now();
  while (true) {
    std::vector<int> need;
    for (int i = 0; i < nb; ++i) {
      if (done[i]) continue;
      ok_grid* G = Gs[i];
      if (!std::isfinite(fn[i])) {
        status[i] = OK_ERR_NONFINITE;
        done[i] = 1;
        continue;
      }
      if (fn[i] <= std::max(G->o.newton_atol, G->o.newton_rtol * r0[i])) {
        ok[i] = 1;
        if (extra[i] >= G->o.newton_extra) {
          done[i] = 1;
          continue;
        }
        ++extra[i];
      }
      if (info[i].newton_its >= G->o.max_newton) {
        done[i] = 1;
        continue;
      }
      need.push_back(i);
    }
    if (need.empty()) break;
    std::vector<ok_grid*> g;
    for (int i : need) {
      assemble_c(Gs[i], Gs[i]->uk);
      g.push_back(Gs[i]);
    }
    std::vector<int> its(need.size(), 0), st(need.size(), OK_SUCCESS);
    std::vector<double> rel(need.size(), 0.0);
    const int prec = Gs[0]->o.precision;
    if (prec == OK_MIXED) {
      std::vector<float*> z;
      for (auto* G : g) z.push_back(G->Zf);
      fgmres_b<float>(g, z, its, rel, st, s);
    } else if (prec == OK_MIXED_HALF) {
      std::vector<__half*> z;
      for (auto* G : g) z.push_back(G->Zh);
      fgmres_b<__half>(g, z, its, rel, st, s);
    } else {
      std::vector<double*> z;
      for (auto* G : g) z.push_back(G->Zd);
      fgmres_b<double>(g, z, its, rel, st, s);
    }
    for (size_t k = 0; k < need.size(); ++k) {
      const int i = need[k];
      ok_grid* G = Gs[i];
      info[i].gmres_its += its[k];
      info[i].last_gmres_its = its[k];
      info[i].rel_resid = rel[k];
      if (st[k] != OK_SUCCESS) {
        status[i] = st[k];
        done[i] = linear_failed[i] = 1;
        continue;
      }
      launch_axpby<double, double>(nv, 1.0, G->xs, 1.0, G->uk, s);
      launch_axpby<double, double>(nv, 1.0, G->xs + nv, 1.0, G->wk, s);
      CKL();
      info[i].newton_its += 1;
      if (rel[k] > G->o.gmres_rtol) {
        status[i] = OK_ERR_NOT_CONVERGED;
        done[i] = linear_failed[i] = 1;
        continue;
      }
      fn[i] = residual(G, G->un, G->wn, G->uk, G->wk, G->f);
    }
  }
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  for (int i = 0; i < nb; ++i) {
    ok_grid* G = Gs[i];
    info[i].newton_resid = fn[i];
    info[i].converged = ok[i];
    info[i].solve_ms = ms;
    if (status[i] == OK_SUCCESS && !ok[i]) status[i] = OK_ERR_NOT_CONVERGED;
    // as ok_timestep: the state is written back after a completed Newton loop
    // (also when it hit its step cap), not after a failed linear solve or a
    // non-finite value
    if (status[i] == OK_SUCCESS || (status[i] == OK_ERR_NOT_CONVERGED && !linear_failed[i])) {
      copy_out(G, u[i], G->uk, nv);
      copy_out(G, w[i], G->wk, nv);
    }
  }
  CK(cudaStreamSynchronize(s));
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

void ok_default_opts(ok_opts* o) {
  if (!o) return;
  o->restart = 30;
  o->max_gmres = 500;
  o->max_newton = 25;
  o->newton_extra = 0;
  o->q_A = 10;
  o->n_V = 5;
  o->k_R = 1;
  o->smooth_pre = 2;
  o->smooth_post = 2;
  o->precision = OK_FP64;
  o->coarse_max = 4;
  o->use_graphs = 1;
  o->fuse_coarse = 1;
  o->tile_fine = 1;
  o->use_pdl = 1;
  o->reorth = 1;
  o->gmres_rtol = 1e-10;
  o->newton_atol = 1e-10;
  o->newton_rtol = 0.0;
  o->smooth_lo_frac = 0.25;
}

const char* ok_last_error(void) { return g_last_error.c_str(); }
const char* ok_version(void) { return "ok-gb300 0.1 (sm_103a)"; }

int ok_grid_create(int dim, int n, const ok_params* p, const ok_opts* o, ok_grid** out) {
  if (!out) {
    g_last_error = "out is NULL";
    return OK_ERR_INVALID_ARG;
  }
  *out = nullptr;
  ok_opts od;
  ok_default_opts(&od);
  if (o) od = *o;
  ok_grid* G = nullptr;
  int st = guarded([&] {
    validate(dim, n, p, &od);
    std::vector<int> sizes = level_sizes(n, od.coarse_max);
    G = new ok_grid();
    G->dim = dim;
    G->n = n;
    G->p = *p;
    G->o = od;
    CK(cudaGetDevice(&G->device));
    CK(cudaDeviceGetAttribute(&G->sms, cudaDevAttrMultiProcessorCount, G->device));
    G->g0 = make_geom(dim, n);
    G->n_levels = (int)sizes.size();
    const double h = 1.0 / n;
    const int fact = dim == 2 ? 2 : 6;
    ResidualCoefs& rc = G->rc;
    rc.a11 = 1.0 + p->dt * p->theta * p->sigma;
    rc.bn = 1.0 - p->dt * (1.0 - p->theta) * p->sigma;
    rc.dsm = p->dt * p->sigma * p->m;
    rc.dth = p->dt * p->theta;
    rc.dth1 = p->dt * (1.0 - p->theta);
    rc.hd = std::pow(h, dim);
    rc.hk = std::pow(h, dim - 2);
    rc.eps2 = p->eps * p->eps;
    rc.vol = rc.hd / fact;
    rc.a4 = dim == 2 ? 2.0 / 720.0 : 6.0 / 5040.0;     // d!/(d+4)!
    rc.a2 = dim == 2 ? 2.0 / 24.0 : 6.0 / 120.0;       // d!/(d+2)!
    JCoefs& jc = G->jc;
    jc.a11hd = rc.a11 * rc.hd;
    jc.dthhk = rc.dth * rc.hk;
    jc.hd = rc.hd;
    jc.alpha = 1.0;
    jc.beta = 0.0;
    CK(cudaStreamCreateWithFlags(&G->s, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&G->ev_in, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&G->ev_out, cudaEventDisableTiming));
    const int NOFF = dim == 2 ? Topo<2>::NOFF : Topo<3>::NOFF;
    const int NCLASS = dim == 2 ? Topo<2>::NCLASS : Topo<3>::NCLASS;
    const int NSLOT = dim == 2 ? Topo<2>::NSLOT : Topo<3>::NSLOT;
    std::vector<double> refM(NCLASS * NOFF), refK(NCLASS * NOFF);
    reference_tables(dim, refM.data(), refK.data());
    rc.msum4 = 0.0;
    if (dim == 2)
      for (int o = 0; o < NOFF; ++o) rc.msum4 += refM[4 * NOFF + o];
    Arena& A = G->arena;
    G->refWM = A.alloc<double>(refM.size());
    G->refWK = A.alloc<double>(refK.size());
    CK(cudaMemcpy(G->refWM, refM.data(), refM.size() * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(G->refWK, refK.data(), refK.size() * sizeof(double), cudaMemcpyHostToDevice));
    {
      std::vector<double> t(NCLASS * NOFF), dv(NCLASS);
      for (int i = 0; i < NCLASS * NOFF; ++i) t[i] = rc.hd * refM[i];
      for (int c = 0; c < NCLASS; ++c) dv[c] = 1.0 / t[c * NOFF];
      G->WM0d = A.alloc<double>(t.size());
      G->dinvM0d = A.alloc<double>(dv.size());
      CK(cudaMemcpy(G->WM0d, t.data(), t.size() * sizeof(double), cudaMemcpyHostToDevice));
      CK(cudaMemcpy(G->dinvM0d, dv.data(), dv.size() * sizeof(double), cudaMemcpyHostToDevice));
      cheb_coefs(0.5, 0.5 * (dim + 2), 60, G->cI1, G->cI2, G->cheb_init_th);
    }
    const long long nv = G->g0.nv, N = 2 * nv;
    G->un = A.alloc<double>(nv);
    G->wn = A.alloc<double>(nv);
    G->uk = A.alloc<double>(nv);
    G->wk = A.alloc<double>(nv);
    G->f = A.alloc<double>(N);
    G->xs = A.alloc<double>(N);
    G->rv = A.alloc<double>(N);
    G->tmp = A.alloc<double>(N);
    G->coef = A.alloc<double>(NSLOT * nv);
    G->coef32 = A.alloc<float>(NSLOT * nv);
    G->V = A.alloc<double>((size_t)(od.restart + 1) * N);
    if (od.precision == OK_MIXED) G->Zf = A.alloc<float>((size_t)od.restart * N);
    else if (od.precision == OK_MIXED_HALF) G->Zh = A.alloc<__half>((size_t)od.restart * N);
    else G->Zd = A.alloc<double>((size_t)od.restart * N);
    G->ks = (KrylovState*)A.alloc<char>(krylov_state_bytes());
    CK(cudaMemset(G->ks, 0, krylov_state_bytes()));
    G->rs.partials = A.alloc<double>((size_t)RED_MAX_BLOCKS * KRYLOV_MAX);
    G->rs.counter = A.alloc<unsigned int>(1);
    CK(cudaMemset(G->rs.counter, 0, sizeof(unsigned int)));
    G->dsc = A.alloc<double>(8);
    G->dflag = A.alloc<int>(1);
    void* hp = nullptr;
    CK(cudaMallocHost(&hp, 64));
    G->hpin = (double*)hp;
    if (od.precision != OK_FP64) {
      build_prec<float>(G, G->pf, sizes, refM, refK);
      G->pf.coef = G->coef32;
      G->pf.tm.coef = G->coef32;
    } else {
      build_prec<double>(G, G->pd, sizes, refM, refK);
      G->pd.coef = G->coef;
      G->pd.tm.coef = G->coef;
    }
    G->graphs.assign(od.restart, nullptr);
    G->cgraphs.assign(od.restart, nullptr);
    G->cgraph_kernels.assign(od.restart, 0);
    G->graph_kernels.assign(od.restart, 0);
    G->graph_tags.assign(od.restart, TagSet{});
    G->pd.prof = &G->prof;
    G->pf.prof = &G->prof;
    krylov_blocks();
    CK(cudaStreamSynchronize(0));      // setup work of this handle (legacy stream); other handles keep running
  });
  if (st != OK_SUCCESS) {
    if (G) ok_grid_destroy(G);
    return st;
  }
  *out = G;
  return OK_SUCCESS;
}

int ok_grid_destroy(ok_grid* G) {
  if (!G) return OK_SUCCESS;
  if (G->s) cudaStreamSynchronize(G->s);
  delete G->ew;                        // its device memory belongs to the arena below
  for (auto& ge : G->graphs)
    if (ge) cudaGraphExecDestroy(ge);
  for (auto& ge : G->cgraphs)
    if (ge) cudaGraphExecDestroy(ge);
  G->prof.destroy();
  G->arena.release();
  if (G->hpin) cudaFreeHost(G->hpin);
  if (G->ev_in) cudaEventDestroy(G->ev_in);
  if (G->ev_out) cudaEventDestroy(G->ev_out);
  if (G->s) cudaStreamDestroy(G->s);
  delete G;
  return OK_SUCCESS;
}

int ok_grid_query(const ok_grid* G, long long* n_vertices, int* n_levels, long long* device_bytes) {
  if (!G) {
    g_last_error = "NULL handle";
    return OK_ERR_INVALID_ARG;
  }
  if (n_vertices) *n_vertices = G->g0.nv;
  if (n_levels) *n_levels = G->n_levels;
  if (device_bytes) *device_bytes = (long long)G->arena.bytes;
  return OK_SUCCESS;
}

int ok_init_w(ok_grid* G, const double* u0, double* w0, ok_stream stream) {
  if (!G || !u0 || !w0) {
    g_last_error = "NULL argument";
    return OK_ERR_INVALID_ARG;
  }
  return guarded([&] {
    StreamScope sc(G, (cudaStream_t)stream);
    const long long nv = G->g0.nv;
    const double* u = stage_in(G, u0, G->uk, nv);
    check_finite(G, u, nv, "u0");
    double* rhs = G->f;
    launch_initw_rhs(G->dim, G->g0, G->refWK, G->rc, u, rhs, G->s);
    CKL();
    // M w0 = rhs by 60 Chebyshev--Jacobi steps on M (contraction <= 0.39 per step)
    Prec<double> tmp;
    tmp.dim = G->dim;
    tmp.cheb<double, double>(G->g0, G->WM0d, G->dinvM0d, rhs, true, G->wk, G->f + nv, G->xs, G->xs + nv, 60,
                             G->cheb_init_th, G->cI1, G->cI2, (double*)nullptr, 1.0, false, G->s);
    CKL();
    copy_out(G, w0, G->wk, nv);
    CK(cudaStreamSynchronize(G->s));
  });
}

int ok_assemble_rhs(ok_grid* G, const double* u_n, const double* w_n, const double* u_k, const double* w_k,
                    double* f, double* norm_out, ok_stream stream) {
  if (!G || !f) {
    g_last_error = "NULL argument";
    return OK_ERR_INVALID_ARG;
  }
  return guarded([&] {
    StreamScope sc(G, (cudaStream_t)stream);
    const long long nv = G->g0.nv;
    const double* un = stage_in(G, u_n, G->un, nv);
    const double* wn = stage_in(G, w_n, G->wn, nv);
    const double* uk = stage_in(G, u_k, G->uk, nv);
    const double* wk = stage_in(G, w_k, G->wk, nv);
    double* fd = is_device_ptr(f) ? f : G->f;
    double nrm = residual(G, un, wn, uk, wk, fd);
    if (fd != f) copy_out(G, f, fd, 2 * nv);
    CK(cudaStreamSynchronize(G->s));
    if (norm_out) *norm_out = nrm;
    if (!std::isfinite(nrm)) fail(OK_ERR_NONFINITE, "non-finite residual");
  });
}

int ok_apply_jacobian(ok_grid* G, const double* u_k, const double* z, double* y, ok_stream stream) {
  if (!G || !y) {
    g_last_error = "NULL argument";
    return OK_ERR_INVALID_ARG;
  }
  return guarded([&] {
    StreamScope sc(G, (cudaStream_t)stream);
    const long long nv = G->g0.nv;
    const double* uk = stage_in(G, u_k, G->uk, nv);
    const double* zd = stage_in(G, z, G->tmp, 2 * nv);
    assemble_c(G, uk);
    double* yd = is_device_ptr(y) ? y : G->rv;
    launch_apply_j<double>(G->dim, G->g0, G->refWM, G->refWK, G->jc, G->coef, zd, yd, nullptr, G->s);
    CKL();
    if (yd != y) copy_out(G, y, yd, 2 * nv);
    CK(cudaStreamSynchronize(G->s));
  });
}

int ok_apply_preconditioner(ok_grid* G, const double* u_k, const double* v, double* z, ok_stream stream) {
  if (!G || !z) {
    g_last_error = "NULL argument";
    return OK_ERR_INVALID_ARG;
  }
  return guarded([&] {
    StreamScope sc(G, (cudaStream_t)stream);
    const long long nv = G->g0.nv;
    const double* uk = stage_in(G, u_k, G->uk, nv);
    const double* vd = stage_in(G, v, G->tmp, 2 * nv);
    assemble_c(G, uk);
    double* zd = is_device_ptr(z) ? z : G->rv;
    precond<double>(G, vd, zd, G->s);
    CKL();
    if (zd != z) copy_out(G, z, zd, 2 * nv);
    CK(cudaStreamSynchronize(G->s));
  });
}

int ok_solve_linear(ok_grid* G, const double* u_k, const double* f, double* x, ok_step_info* info,
                    ok_stream stream) {
  if (!G || !x) {
    g_last_error = "NULL argument";
    return OK_ERR_INVALID_ARG;
  }
  return guarded([&] {
    StreamScope sc(G, (cudaStream_t)stream);
    const long long nv = G->g0.nv;
    const double* uk = stage_in(G, u_k, G->uk, nv);
    const double* fd = stage_in(G, f, G->f, 2 * nv);
    check_finite(G, fd, 2 * nv, "f");
    assemble_c(G, uk);
    auto t0 = std::chrono::steady_clock::now();
    int its = 0;
    double rel = 0;
    double* xd = is_device_ptr(x) ? x : G->xs;
    linear_solve(G, fd, xd, its, rel);
    if (xd != x) copy_out(G, x, xd, 2 * nv);
    CK(cudaStreamSynchronize(G->s));
    if (info) {
      std::memset(info, 0, sizeof(*info));
      info->gmres_its = its;
      info->last_gmres_its = its;
      info->rel_resid = rel;
      info->converged = rel <= G->o.gmres_rtol;
      info->solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    if (rel > G->o.gmres_rtol) fail(OK_ERR_NOT_CONVERGED, "FGMRES did not reach gmres_rtol within max_gmres");
  });
}

int ok_newton_step(ok_grid* G, const double* u_n, const double* w_n, double* u_k, double* w_k,
                   ok_step_info* info, ok_stream stream) {
  if (!G || !u_k || !w_k) {
    g_last_error = "NULL argument";
    return OK_ERR_INVALID_ARG;
  }
  ok_step_info loc;
  std::memset(&loc, 0, sizeof(loc));
  int st = guarded([&] {
    StreamScope sc(G, (cudaStream_t)stream);
    const long long nv = G->g0.nv;
    const double* un = stage_in(G, u_n, G->un, nv);
    const double* wn = stage_in(G, w_n, G->wn, nv);
    if (un != G->un) CK(cudaMemcpyAsync(G->un, un, nv * sizeof(double), cudaMemcpyDeviceToDevice, G->s));
    if (wn != G->wn) CK(cudaMemcpyAsync(G->wn, wn, nv * sizeof(double), cudaMemcpyDeviceToDevice, G->s));
    CK(cudaMemcpyAsync(G->uk, u_k, nv * sizeof(double), cudaMemcpyDefault, G->s));
    CK(cudaMemcpyAsync(G->wk, w_k, nv * sizeof(double), cudaMemcpyDefault, G->s));
    check_finite(G, G->uk, nv, "u_k");
    check_finite(G, G->wk, nv, "w_k");
    double r0 = residual(G, G->un, G->wn, G->uk, G->wk, G->f);
    loc.newton_resid0 = r0;
    if (!std::isfinite(r0)) fail(OK_ERR_NONFINITE, "non-finite residual");
    double ms = 0;
    newton_update(G, loc, ms);
    loc.solve_ms = ms;
    loc.newton_resid = residual(G, G->un, G->wn, G->uk, G->wk, G->f);
    loc.converged = loc.newton_resid <= std::max(G->o.newton_atol, G->o.newton_rtol * r0);
    copy_out(G, u_k, G->uk, nv);
    copy_out(G, w_k, G->wk, nv);
    CK(cudaStreamSynchronize(G->s));
  });
  if (info) *info = loc;
  return st;
}

int ok_timestep(ok_grid* G, double* u, double* w, ok_step_info* info, ok_stream stream) {
  if (!G || !u || !w) {
    g_last_error = "NULL argument";
    return OK_ERR_INVALID_ARG;
  }
  ok_step_info loc;
  std::memset(&loc, 0, sizeof(loc));
  int st = guarded([&] {
    StreamScope sc(G, (cudaStream_t)stream);
    const long long nv = G->g0.nv;
    CK(cudaMemcpyAsync(G->un, u, nv * sizeof(double), cudaMemcpyDefault, G->s));
    CK(cudaMemcpyAsync(G->wn, w, nv * sizeof(double), cudaMemcpyDefault, G->s));
    check_finite(G, G->un, nv, "u");
    check_finite(G, G->wn, nv, "w");
    CK(cudaMemcpyAsync(G->uk, G->un, nv * sizeof(double), cudaMemcpyDeviceToDevice, G->s));
    CK(cudaMemcpyAsync(G->wk, G->wn, nv * sizeof(double), cudaMemcpyDeviceToDevice, G->s));
    double fn = residual(G, G->un, G->wn, G->uk, G->wk, G->f);
    const double r0 = fn;
    loc.newton_resid0 = r0;
    int extra = 0;
    double ms = 0;
    bool ok = false;
    while (true) {
      if (!std::isfinite(fn)) fail(OK_ERR_NONFINITE, "non-finite Newton residual");
      if (fn <= std::max(G->o.newton_atol, G->o.newton_rtol * r0)) {
        ok = true;
        if (extra >= G->o.newton_extra) break;
        ++extra;
      }
      if (loc.newton_its >= G->o.max_newton) break;
      newton_update(G, loc, ms);
      fn = residual(G, G->un, G->wn, G->uk, G->wk, G->f);
    }
    loc.newton_resid = fn;
    loc.converged = ok;
    loc.solve_ms = ms;
    copy_out(G, u, G->uk, nv);
    copy_out(G, w, G->wk, nv);
    CK(cudaStreamSynchronize(G->s));
    if (!ok) fail(OK_ERR_NOT_CONVERGED, "Newton did not converge within max_newton steps");
  });
  if (info) *info = loc;
  return st;
}

int ok_profile(ok_grid* G, int enable) {
  if (!G) {
    g_last_error = "NULL handle";
    return OK_ERR_INVALID_ARG;
  }
  return guarded([&] {
    CK(cudaStreamSynchronize(G->s));
    const bool on = enable != 0;
    if (on != G->prof.on) {            // graphs are re-captured with/without the event nodes
      for (auto& ge : G->graphs)
        if (ge) cudaGraphExecDestroy(ge), ge = nullptr;
    }
    if (on) G->prof.create();
    G->prof.on = on;
    for (int t = 0; t < PT_COUNT; ++t) {
      if (on) G->prof.samples[t] = 0, G->prof.total_ms[t] = 0.0;
    }
  });
}

int ok_profile_read(const ok_grid* G, ok_kernel_stat* out, int max, int* count) {
  if (!G || (max > 0 && !out)) {
    g_last_error = "NULL argument";
    return OK_ERR_INVALID_ARG;
  }
  int n = 0;
  for (int t = 0; t < PT_COUNT && n < max; ++t, ++n) {
    std::memset(&out[n], 0, sizeof(ok_kernel_stat));
    std::strncpy(out[n].name, kProfNames[t], sizeof(out[n].name) - 1);
    out[n].samples = G->prof.samples[t];
    out[n].total_ms = G->prof.total_ms[t];
  }
  if (count) *count = n;
  return OK_SUCCESS;
}

int ok_arnoldi_hessenberg(ok_grid* G, double* H, int ldh, int max_k, int* k, ok_stream stream) {
  if (!G || !k || max_k < 0 || (max_k > 0 && !H) || ldh < max_k + 1) {
    g_last_error = "NULL argument, max_k < 0 or ldh < max_k + 1";
    return OK_ERR_INVALID_ARG;
  }
  return guarded([&] {
    StreamScope sc(G, (cudaStream_t)stream);
    double steps = 0.0;
    CK(cudaMemcpyAsync(&steps, ks_nsteps_ptr(G->ks), sizeof(double), cudaMemcpyDeviceToHost, G->s));
    CK(cudaStreamSynchronize(G->s));
    // the leading columns of Hbar are themselves the Arnoldi matrix of fewer steps
    const int kk = std::max(0, std::min({(int)steps, max_k, KRYLOV_MAX - 1}));
    const int ld = KRYLOV_MAX + 1;
    std::vector<double> R((size_t)ld * kk), cs(kk), sn(kk);
    if (kk > 0) {
      CK(cudaMemcpyAsync(R.data(), ks_H_ptr(G->ks), R.size() * sizeof(double), cudaMemcpyDeviceToHost, G->s));
      CK(cudaMemcpyAsync(cs.data(), ks_cs_ptr(G->ks), kk * sizeof(double), cudaMemcpyDeviceToHost, G->s));
      CK(cudaMemcpyAsync(sn.data(), ks_sn_ptr(G->ks), kk * sizeof(double), cudaMemcpyDeviceToHost, G->s));
      CK(cudaStreamSynchronize(G->s));
    }
    for (int j = 0; j < kk; ++j)
      for (int i = 0; i <= kk; ++i) H[(size_t)ldh * j + i] = i <= j ? R[(size_t)ld * j + i] : 0.0;
    if (ok_givens_unrotate(kk, H, ldh, cs.data(), sn.data()) != OK_SUCCESS)
      fail(OK_ERR_INVALID_ARG, "Givens restoration rejected its arguments");
    *k = kk;
  });
}

int ok_ritz_values(ok_grid* G, double* re, double* im, int max, int* count, ok_stream stream) {
  if (!G || !count || max < 0 || (max > 0 && (!re || !im))) {
    g_last_error = "NULL argument or max < 0";
    return OK_ERR_INVALID_ARG;
  }
  const int cap = std::min(max, KRYLOV_MAX - 1);
  std::vector<double> H((size_t)(cap + 1) * std::max(cap, 1));
  int k = 0;
  int st = ok_arnoldi_hessenberg(G, H.data(), cap + 1, cap, &k, stream);
  if (st != OK_SUCCESS) return st;
  st = ok_hessenberg_eigenvalues(k, H.data(), cap + 1, re, im);
  if (st != OK_SUCCESS) {
    g_last_error = st == OK_ERR_NONFINITE ? "non-finite Arnoldi matrix"
                   : st == OK_ERR_NOMEM    ? "host allocation failed"
                                           : "QR iteration did not converge";
    return st;
  }
  *count = k;
  g_last_error.clear();
  return OK_SUCCESS;
}

int ok_tuning_save(const char* path) {
  if (!path) {
    g_last_error = "NULL path";
    return OK_ERR_INVALID_ARG;
  }
  FILE* f = std::fopen(path, "w");
  if (!f) {
    g_last_error = std::string("cannot write ") + path;
    return OK_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(g_tune_mu);
  std::fprintf(f, "# ok-gb300 autotuner choices: dim n bytes-per-value choice\n");
  for (const auto& kv : g_tune) std::fprintf(f, "%d %d %d %d\n", kv.first[1], kv.first[2], kv.first[3], kv.second);
  std::fclose(f);
  g_last_error.clear();
  return OK_SUCCESS;
}

int ok_tuning_load(const char* path) {
  if (!path) {
    g_last_error = "NULL path";
    return OK_ERR_INVALID_ARG;
  }
  FILE* f = std::fopen(path, "r");
  if (!f) {
    g_last_error = std::string("cannot read ") + path;
    return OK_ERR_INVALID_ARG;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    dev = 0;
  }
  char line[256];
  int bad = 0;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  while (std::fgets(line, sizeof(line), f)) {
    if (line[0] == '#' || line[0] == '\n') continue;
    int d = 0, n = 0, b = 0, c = 0;
    if (std::sscanf(line, "%d %d %d %d", &d, &n, &b, &c) == 4 && (d == 2 || d == 3) && n >= 1 &&
        (b == 4 || b == 8) && c >= 0 && c <= (d == 2 ? STRIP_SHAPES - 1 : PLANE_SHAPES))
      g_tune[{dev, d, n, b, 0}] = c;
    else
      ++bad;
  }
  std::fclose(f);
  if (bad) {
    g_last_error = std::to_string(bad) + " malformed line(s) in " + path;
    return OK_ERR_INVALID_ARG;
  }
  g_last_error.clear();
  return OK_SUCCESS;
}

int ok_grid_tuning(const ok_grid* G, int* level_n, int* choice, int max, int* count) {
  if (!G || !count || max < 0 || (max > 0 && (!level_n || !choice))) {
    g_last_error = "NULL argument or max < 0";
    return OK_ERR_INVALID_ARG;
  }
  const auto& t = G->o.precision == OK_FP64 ? G->pd.tuned : G->pf.tuned;
  const int k = std::min<int>(max, (int)t.size());
  for (int i = 0; i < k; ++i) {
    level_n[i] = t[i].first;
    choice[i] = t[i].second;
  }
  *count = k;
  return OK_SUCCESS;
}

int ok_energy(ok_grid* G, const double* u, double* terms, double* E, ok_stream stream) {
  if (!G || !u || (!terms && !E)) {
    g_last_error = "NULL argument";
    return OK_ERR_INVALID_ARG;
  }
  return guarded([&] {
    StreamScope sc(G, (cudaStream_t)stream);
    const long long nv = G->g0.nv;
    const double* ud = stage_in(G, u, G->tmp, nv);
    check_finite(G, ud, nv, "u");
    double t[3];
    energy(G, ud, t);
    if (terms) std::memcpy(terms, t, sizeof(t));
    if (E) *E = t[0] + t[1] + t[2];
    if (G->ew->last_its >= 500) fail(OK_ERR_NOT_CONVERGED, "the energy's Neumann solve did not converge");
  });
}

long long ok_launch_count(void) { return g_launch_count.load(); }

int ok_solve_batch(ok_request* reqs, int count, ok_batch_info* out, ok_stream stream) {
  if (count < 0 || (count > 0 && !reqs)) {
    g_last_error = "invalid batch";
    return OK_ERR_INVALID_ARG;
  }
  auto t0 = std::chrono::steady_clock::now();
  auto now = [&] { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); };
  std::vector<int> valid;
  for (int i = 0; i < count; ++i) {
    ok_request& r = reqs[i];
    r.status = OK_SUCCESS;
    r.newton_its = r.gmres_its = 0;
    r.seconds = 0.0;
    if (!r.grid || !r.u || !r.w || r.steps < 0) r.status = OK_ERR_INVALID_ARG;
    else valid.push_back(i);
  }
  // cohorts: requests on distinct handles of the same grid, options and
  // multigrid structure, at most BATCH_MAX together, in request order
  std::vector<std::vector<int>> cohorts;
  std::vector<int> taken(count, 0);
  for (size_t a = 0; a < valid.size(); ++a) {
    const int i = valid[a];
    if (taken[i]) continue;
    std::vector<int> c{i};
    taken[i] = 1;
    for (size_t b = a + 1; b < valid.size() && (int)c.size() < BATCH_MAX; ++b) {
      const int k = valid[b];
      if (taken[k]) continue;
      bool distinct = true;
      for (int m : c) distinct = distinct && reqs[m].grid != reqs[k].grid;
      if (distinct && cohort_compatible(reqs[i].grid, reqs[k].grid)) {
        c.push_back(k);
        taken[k] = 1;
      }
    }
    cohorts.push_back(c);
  }
  for (const auto& c : cohorts) {
    if (c.size() == 1) {                                  // alone: the timestep path itself
      ok_request& r = reqs[c[0]];
      for (int k = 0; k < r.steps; ++k) {
        ok_step_info info = {};
        const int st = ok_timestep(r.grid, r.u, r.w, &info, stream);
        r.newton_its += info.newton_its;
        r.gmres_its += info.gmres_its;
        if (st != OK_SUCCESS) {
          r.status = st;
          break;
        }
      }
      r.seconds = now();
      continue;
    }
    std::vector<ok_grid*> Gs;
    for (int i : c) Gs.push_back(reqs[i].grid);
    std::string msg;
    const int st = guarded([&] {
      ok_grid* G0 = Gs[0];
      cudaStream_t cs = G0->s;
      // the cohort's stream follows the caller's stream and every member's
      // earlier work; the caller's stream follows the cohort at the end
      CK(cudaEventRecord(G0->ev_in, (cudaStream_t)stream));
      CK(cudaStreamWaitEvent(cs, G0->ev_in, 0));
      for (auto* G : Gs)
        if (G != G0) {
          CK(cudaEventRecord(G->ev_in, G->s));
          CK(cudaStreamWaitEvent(cs, G->ev_in, 0));
        }
      {
        CohortStreams swap(Gs, cs);
        int steps = 0;
        for (int i : c) steps = std::max(steps, reqs[i].steps);
        for (int t = 0; t < steps; ++t) {
          std::vector<ok_grid*> g;
          std::vector<double*> u, w;
          std::vector<int> idx;
          for (int i : c)
            if (reqs[i].status == OK_SUCCESS && t < reqs[i].steps) {
              g.push_back(reqs[i].grid);
              u.push_back(reqs[i].u);
              w.push_back(reqs[i].w);
              idx.push_back(i);
            }
          if (g.empty()) break;
          std::vector<ok_step_info> info(g.size());
          std::vector<int> status(g.size(), OK_SUCCESS);
          timestep_b(g, u.data(), w.data(), info, status, cs);
          for (size_t k = 0; k < idx.size(); ++k) {
            ok_request& r = reqs[idx[k]];
            r.newton_its += info[k].newton_its;
            r.gmres_its += info[k].gmres_its;
            if (status[k] != OK_SUCCESS) r.status = status[k];
            if (status[k] != OK_SUCCESS || t + 1 == r.steps) r.seconds = now();
          }
        }
      }
      CK(cudaEventRecord(G0->ev_out, cs));
      CK(cudaStreamWaitEvent((cudaStream_t)stream, G0->ev_out, 0));
      for (auto* G : Gs)
        if (G != G0) CK(cudaStreamWaitEvent(G->s, G0->ev_out, 0));
    });
    if (st != OK_SUCCESS) {                               // a CUDA or host failure of the cohort itself
      for (int i : c)
        if (reqs[i].status == OK_SUCCESS) reqs[i].status = st, reqs[i].seconds = now();
    }
  }
  int done = 0, failed = 0;
  for (int i = 0; i < count; ++i) (reqs[i].status == OK_SUCCESS ? done : failed) += 1;
  if (out) {
    out->completed = done;
    out->failed = failed;
    out->seconds = now();
  }
  if (failed == 0) return OK_SUCCESS;
  for (int i = 0; i < count; ++i)
    if (reqs[i].status != OK_SUCCESS) {
      g_last_error = "request " + std::to_string(i) + " failed with status " + std::to_string(reqs[i].status);
      return reqs[i].status;
    }
  return OK_SUCCESS;
}

// ---------------------------------------------------------------------------
// serving: continuous admission of whole simulations
// ---------------------------------------------------------------------------
// Device bytes a handle of (dim, n, o) allocates, from the same sizes
// ok_grid_create uses (an upper estimate for admission; the multigrid
// vectors and the coarse inverse are bounded from above).
static long long serve_estimate(int dim, int n, const ok_opts& o) {
  const double nv = std::pow((double)(n + 1), dim);
  const double N = 2.0 * nv;
  const int nslot = dim == 2 ? 4 : 8;
  const double zb = o.precision == OK_FP64 ? 8.0 : (o.precision == OK_MIXED ? 4.0 : 2.0);
  const double tb = o.precision == OK_FP64 ? 8.0 : 4.0;
  double b = 8.0 * N * (o.restart + 1) + zb * N * o.restart;   // V, Z
  b += nslot * nv * 12.0;                                     // C store, float64 + float32
  b += 12.0 * nv * 8.0;                                       // state and work vectors
  b += 9.0 * nv * tb * (dim == 2 ? 4.0 / 3.0 : 8.0 / 7.0);  // multigrid vectors over the levels
  const double nc = std::min(std::pow((double)(o.coarse_max + 2), dim), 4913.0);
  b += nc * nc * (8.0 + 2.0 * tb) + (1 << 20);                // coarse inverse (+ padded copy), scalars
  return b < 9.0e18 ? (long long)b : 9000000000000000000LL;
}

extern "C" int ok_serve(ok_serve_request* reqs, int count, int max_inflight, long long mem_budget,
                        ok_serve_info* info) {
  if (count < 0 || (count > 0 && !reqs) || max_inflight < 1 || mem_budget <= 0) {
    g_last_error = "invalid serving arguments";
    return OK_ERR_INVALID_ARG;
  }
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) {
    cudaGetLastError();
    g_last_error = "no CUDA device";
    return OK_ERR_CUDA;
  }
  PoolScope pool;
  const auto t0 = std::chrono::steady_clock::now();
  auto now = [&] { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); };
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return reqs[a].arrival < reqs[b].arrival; });

  // One group per (dim, n, options): its own host thread and stream run the
  // group's admitted requests in cohorts, a timestep at a time; a request
  // joins at the next timestep after its setup and leaves after its last.
  struct Group {
    std::deque<int> ready;            // set up, waiting to join
    std::vector<int> active;          // stepping
    std::thread th;
  };
  std::mutex mu;
  std::condition_variable cv;
  bool closing = false;
  int inflight = 0, peak_inflight = 0, peak_cohort = 0, cohort_steps = 0;
  long long bytes = 0, peak_bytes = 0;
  std::map<std::string, std::unique_ptr<Group>> groups;
  std::vector<ok_grid*> grid(count, nullptr);
  std::vector<int> steps_done(count, 0);
  std::vector<ok_opts> opts(count);
  std::vector<std::thread> setups;
  setups.reserve(count);

  auto finish = [&](int i, int status) {             // request i leaves: handle freed, slot released
    ok_serve_request& q = reqs[i];
    if (status != OK_SUCCESS && q.message[0] == 0) {
      std::strncpy(q.message, ok_last_error(), sizeof(q.message) - 1);
      q.message[sizeof(q.message) - 1] = 0;
    }
    if (grid[i]) ok_grid_destroy(grid[i]);
    grid[i] = nullptr;
    q.status = status;
    q.t_done = now();
    {
      std::lock_guard<std::mutex> lk(mu);
      --inflight;
      bytes -= q.device_bytes;
    }
    cv.notify_all();
  };

  auto group_loop = [&](Group* G) {
    cudaSetDevice(device);
    cudaStream_t gs = nullptr;
    if (cudaStreamCreateWithFlags(&gs, cudaStreamNonBlocking) != cudaSuccess) gs = nullptr;
    while (true) {
      {
        std::unique_lock<std::mutex> lk(mu);
        cv.wait(lk, [&] { return !G->ready.empty() || !G->active.empty() || closing; });
        // members join while the cohort has room and shares launches with them
        for (auto it = G->ready.begin(); it != G->ready.end() && (int)G->active.size() < BATCH_MAX;) {
          if (G->active.empty() || cohort_compatible(grid[G->active[0]], grid[*it])) {
            G->active.push_back(*it);
            it = G->ready.erase(it);
          } else {
            ++it;
          }
        }
        if (G->active.empty() && G->ready.empty() && closing) break;
        if (G->active.empty()) continue;
      }
      std::vector<int> act = G->active;
      {
        std::lock_guard<std::mutex> lk(mu);
        peak_cohort = std::max(peak_cohort, (int)act.size());
        if (act.size() > 1) ++cohort_steps;
      }
      std::vector<int> status(act.size(), OK_SUCCESS);
      std::vector<ok_step_info> si(act.size());
      if (!gs) {
        for (size_t k = 0; k < act.size(); ++k) status[k] = OK_ERR_CUDA;
      } else if (act.size() == 1) {
        status[0] = ok_timestep(grid[act[0]], reqs[act[0]].u, reqs[act[0]].w, &si[0], (ok_stream)gs);
      } else {
        std::vector<ok_grid*> Gs;
        std::vector<double*> u, w;
        for (int i : act) Gs.push_back(grid[i]), u.push_back(reqs[i].u), w.push_back(reqs[i].w);
        const int st = guarded([&] {
          CohortStreams swap(Gs, gs);
          timestep_b(Gs, u.data(), w.data(), si, status, gs);
        });
        if (st != OK_SUCCESS)
          for (auto& x : status)
            if (x == OK_SUCCESS) x = st;
      }
      std::vector<int> keep;
      for (size_t k = 0; k < act.size(); ++k) {
        const int i = act[k];
        reqs[i].newton_its += si[k].newton_its;
        reqs[i].gmres_its += si[k].gmres_its;
        if (status[k] != OK_SUCCESS) {
          finish(i, status[k]);
        } else if (++steps_done[i] >= reqs[i].steps) {
          finish(i, OK_SUCCESS);
        } else {
          keep.push_back(i);
        }
      }
      std::lock_guard<std::mutex> lk(mu);
      G->active = keep;
    }
    if (gs) cudaStreamDestroy(gs);
  };

  // validation; the valid requests in arrival order
  std::vector<int> valid;
  for (int i : order) {
    ok_serve_request& r = reqs[i];
    r.status = OK_SUCCESS;
    r.newton_its = r.gmres_its = 0;
    r.t_admit = r.t_done = 0.0;
    r.message[0] = 0;
    ok_default_opts(&opts[i]);
    if (r.opts) opts[i] = *r.opts;
    const ok_opts& o = opts[i];
    r.device_bytes = 0;
    if (!r.u || !r.w || r.steps < 0 || r.dim < 2 || r.dim > 3 || r.n < 2 || o.restart < 1 ||
        o.restart >= KRYLOV_MAX || o.coarse_max < 1) {
      r.status = OK_ERR_INVALID_ARG;
      continue;
    }
    r.device_bytes = serve_estimate(r.dim, r.n, o);
    if (r.device_bytes > mem_budget) {
      r.status = OK_ERR_NOMEM;
      continue;
    }
    valid.push_back(i);
  }
  // Admission.  A request is admitted once fewer than max_inflight are in
  // flight and its estimate fits the budget beside theirs; a younger request
  // that fits may pass an older one that waits for memory, unless the oldest
  // waiting request has waited HOL_WAIT seconds (then it alone may enter, so
  // it cannot starve while small requests keep arriving).
  constexpr double HOL_WAIT = 1.0;
  auto admit = [&](int i) {
    ok_serve_request& r = reqs[i];
    const ok_opts& o = opts[i];
    r.t_admit = now();
    // the group of (dim, n, options): started on first use
    std::string key(reinterpret_cast<const char*>(&o), sizeof(ok_opts));
    key += std::to_string(r.dim) + "/" + std::to_string(r.n);
    Group* G = nullptr;
    {
      std::lock_guard<std::mutex> lk(mu);
      auto& slot = groups[key];
      if (!slot) {
        slot.reset(new Group());
        try {
          slot->th = std::thread(group_loop, slot.get());
        } catch (const std::exception&) {
          slot.reset();
        }
      }
      G = slot.get();
    }
    if (!G) {
      std::strncpy(r.message, "could not start a group thread", sizeof(r.message) - 1);
      std::lock_guard<std::mutex> lk(mu);
      --inflight;
      bytes -= r.device_bytes;
      r.status = OK_ERR_NOMEM;
      r.t_done = now();
      groups.erase(key);
      return;
    }
    try {
      setups.emplace_back([&, i, G] {                   // handle and w0 on the request's own thread
        ok_serve_request& q = reqs[i];
        cudaSetDevice(device);
        cudaStream_t st = nullptr;
        int status = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess ? OK_SUCCESS : OK_ERR_CUDA;
        if (status == OK_SUCCESS) status = ok_grid_create(q.dim, q.n, &q.params, &opts[i], &grid[i]);
        if (status == OK_SUCCESS && q.init_w) status = ok_init_w(grid[i], q.u, q.w, (ok_stream)st);
        if (st) cudaStreamDestroy(st);
        if (status != OK_SUCCESS || q.steps == 0) {
          finish(i, status);
          return;
        }
        {
          std::lock_guard<std::mutex> lk(mu);
          G->ready.push_back(i);
        }
        cv.notify_all();
      });
    } catch (const std::exception&) {
      std::strncpy(r.message, "could not start a setup thread", sizeof(r.message) - 1);
      finish(i, OK_ERR_NOMEM);
    }
  };
  std::deque<int> waiting;                            // arrived, not yet admitted, in arrival order
  size_t next = 0;                                    // next valid request still to arrive
  while (next < valid.size() || !waiting.empty()) {
    int pick = -1;
    {
      std::unique_lock<std::mutex> lk(mu);
      const double t = now();
      while (next < valid.size() && reqs[valid[next]].arrival <= t) waiting.push_back(valid[next++]);
      if (inflight < max_inflight && !waiting.empty()) {
        const bool head_may_be_passed = t - reqs[waiting.front()].arrival < HOL_WAIT;
        for (size_t k = 0; k < waiting.size(); ++k) {
          if (bytes + reqs[waiting[k]].device_bytes <= mem_budget) {
            pick = (int)k;
            break;
          }
          if (!head_may_be_passed) break;
        }
      }
      if (pick < 0) {                                 // wait for a request to finish or to arrive
        double dt = 0.05;
        if (next < valid.size()) dt = std::min(dt, std::max(0.0, reqs[valid[next]].arrival - t));
        cv.wait_for(lk, std::chrono::duration<double>(dt));
        continue;
      }
      const int i = waiting[pick];
      waiting.erase(waiting.begin() + pick);
      ++inflight;
      bytes += reqs[i].device_bytes;
      peak_inflight = std::max(peak_inflight, inflight);
      peak_bytes = std::max(peak_bytes, bytes);
      pick = i;
    }
    admit(pick);
  }
  for (auto& t : setups) t.join();
  {
    std::lock_guard<std::mutex> lk(mu);
    closing = true;
  }
  cv.notify_all();
  for (auto& kv : groups)
    if (kv.second && kv.second->th.joinable()) kv.second->th.join();
  int done = 0, failed = 0;
  for (int i = 0; i < count; ++i) (reqs[i].status == OK_SUCCESS ? done : failed) += 1;
  if (info) {
    info->completed = done;
    info->failed = failed;
    info->peak_inflight = peak_inflight;
    info->peak_bytes = peak_bytes;
    info->seconds = now();
    info->peak_cohort = peak_cohort;
    info->cohort_steps = cohort_steps;
  }
  for (int i = 0; i < count; ++i)
    if (reqs[i].status != OK_SUCCESS) {
      g_last_error = "request " + std::to_string(i) + " failed with status " + std::to_string(reqs[i].status);
      return reqs[i].status;
    }
  return OK_SUCCESS;
}

}  // extern "C"

// Lets other translation units set the message ok_last_error() returns.
void okg::set_last_error(const char* msg) { g_last_error = msg; }
