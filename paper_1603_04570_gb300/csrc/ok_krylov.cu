// ok_krylov.cu -- float64 kernels of right-preconditioned restarted FGMRES.
//
// Arnoldi step j (Saad, "A flexible inner-outer preconditioned GMRES
// algorithm", SISC 14, 1993) with w = J z_j orthogonalised against
// v_0..v_j by classical Gram--Schmidt with re-orthogonalisation:
//     h1 = V^T w;  w -= V h1;  [h2 = V^T w;  w -= V h2;]  H(:,j) = h1 (+ h2);
//     eta = ||w||;  H(j+1,j) = eta;  v_{j+1} = w / eta;
// the bracketed second pass runs always (CGS2), never (one classical pass), or,
// by the criterion of Daniel, Gragg, Kaufman and Stewart (Math. Comp. 30,
// 1976), only when the first pass cancelled more than half of ||w||^2
// (||w_1||^2 < ||w_0||^2 / 2); that decision is taken on the device and the
// second-pass kernels return at once when it is not needed.  The new column is then reduced by Givens
// rotations and |g_{j+1}| is the residual norm of the least-squares problem
// min || beta e_1 - H y ||.
//
// Reductions are deterministic: a fixed grid, a fixed element-to-thread map,
// per-block partials and an in-order sum by the last block to finish (found
// with an atomic ticket; no block waits on another).
#include <math.h>
#include "ok_internal.cuh"
#include "ok_kernels.h"

namespace okg {

struct KrylovState {
  double H[(KRYLOV_MAX + 1) * KRYLOV_MAX];   // H(i,j) at i + (KRYLOV_MAX+1) j; rotated in place
  double cs[KRYLOV_MAX], sn[KRYLOV_MAX];
  double g[KRYLOV_MAX + 1];
  double h1[KRYLOV_MAX + 1], h2[KRYLOV_MAX + 1];
  double y[KRYLOV_MAX];
  double beta, inv_beta;
  double eta, inv_eta;
  double resid;
  double go;          // 1 while the cycle continues: set by each step (read with eta..nsteps)
  double nsteps;      // Arnoldi steps taken in this cycle
  double thresh;      // the steps' stop test: resid <= thresh (rtol ||f||)
  double nw0;         // ||w||^2 before the first Gram--Schmidt pass
  int skip2;          // 1: the second pass is not needed this step
  int passes2;        // second passes taken since the handle was created
};

size_t krylov_state_bytes() { return sizeof(KrylovState); }
double* ks_resid_ptr(KrylovState* ks) { return &ks->resid; }
double* ks_eta_ptr(KrylovState* ks) { return &ks->eta; }
double* ks_beta_ptr(KrylovState* ks) { return &ks->beta; }
double* ks_h1_ptr(KrylovState* ks) { return ks->h1; }
double* ks_h2_ptr(KrylovState* ks) { return ks->h2; }
int* ks_skip2_ptr(KrylovState* ks) { return &ks->skip2; }
double* ks_nw0_ptr(KrylovState* ks) { return &ks->nw0; }
int* ks_passes2_ptr(KrylovState* ks) { return &ks->passes2; }
const double* ks_H_ptr(const KrylovState* ks) { return ks->H; }
const double* ks_cs_ptr(const KrylovState* ks) { return ks->cs; }
const double* ks_sn_ptr(const KrylovState* ks) { return ks->sn; }
const double* ks_nsteps_ptr(const KrylovState* ks) { return &ks->nsteps; }

static constexpr int RT = 256;    // threads per reduction block
static constexpr int KC = 16;     // vectors per multi-dot launch (register budget)

// reduction grid per device (4 blocks per SM), looked up once per device
static constexpr int KB_MAX_DEVICES = 64;
static std::atomic<int> g_blocks[KB_MAX_DEVICES];
int krylov_blocks() {
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= KB_MAX_DEVICES) dev = 0;
  int b = g_blocks[dev].load(std::memory_order_relaxed);
  if (b == 0) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    b = sms > 0 ? 4 * sms : 512;
    if (b > RED_MAX_BLOCKS) b = RED_MAX_BLOCKS;
    g_blocks[dev].store(b, std::memory_order_relaxed);
  }
  return b;
}

// Reduce acc[0..K) over the block into partials[blockIdx.x * KRYLOV_MAX + k].
template <int NK>
__device__ __forceinline__ void block_partials(const double (&acc)[NK], int K, double* __restrict__ partials) {
  __shared__ double sm[RT / 32][NK];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NK; ++k) {
    if (k < K) {
      double a = acc[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      if (lane == 0) sm[warp][k] = a;
    }
  }
  __syncthreads();
  if (threadIdx.x < K) {
    double a = 0.0;
#pragma unroll
    for (int w = 0; w < RT / 32; ++w) a += sm[w][threadIdx.x];
    partials[blockIdx.x * KRYLOV_MAX + threadIdx.x] = a;
  }
}

// True in exactly one block: the last to finish.  Resets the ticket.
__device__ __forceinline__ bool last_block(unsigned int* counter) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int t = atomicAdd(counter, 1u);
    last = (t == gridDim.x - 1);
    if (last) *counter = 0u;
  }
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// Sum of the per-block partials of value k, by one warp: lane-strided over the
// blocks, then an xor-shuffle tree (a fixed order, so results are reproducible).
__device__ __forceinline__ double warp_sum_partials(const double* __restrict__ partials, int k) {
  const int lane = threadIdx.x & 31;
  double a = 0.0;
  for (int b = lane; b < (int)gridDim.x; b += 32) a += partials[b * KRYLOV_MAX + k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  return a;
}

__device__ __forceinline__ void final_sums(const double* __restrict__ partials, int K, double* __restrict__ out) {
  const int warp = threadIdx.x >> 5;
  for (int k = warp; k < K; k += RT / 32) {
    const double a = warp_sum_partials(partials, k);
    if ((threadIdx.x & 31) == 0) out[k] = a;
  }
}

// The multi-dot and update kernels take the number of basis vectors K
// (<= KC) as a template argument, so that every V load of an element is
// unconditional and can be in flight at once.
// out[k] = v_k . w (k < K); with NORM also *nrm = w . w.  A kernel given a
// skip flag returns at once when the flag is set.
template <int K, bool NORM>
__device__ __forceinline__ void multidot_body(const double* __restrict__ V, long long ldv,
                                              const double* __restrict__ w, long long N,
                                              double* __restrict__ partials, unsigned int* counter,
                                              double* __restrict__ out, const int* __restrict__ skip,
                                              double* __restrict__ nrm) {
  if (skip && *skip) return;
  constexpr int NA = K + (NORM ? 1 : 0);
  double acc[NA];
#pragma unroll
  for (int k = 0; k < NA; ++k) acc[k] = 0.0;
  for (long long e = blockIdx.x * (long long)RT + threadIdx.x; e < N; e += (long long)gridDim.x * RT) {
    const double we = w[e];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = fma(V[k * ldv + e], we, acc[k]);
    if constexpr (NORM) acc[K] = fma(we, we, acc[K]);
  }
  block_partials<NA>(acc, NA, partials);
  if (!last_block(counter)) return;
  const int warp = threadIdx.x >> 5;
  for (int k = warp; k < NA; k += RT / 32) {
    const double a = warp_sum_partials(partials, k);
    if ((threadIdx.x & 31) == 0) {
      if (k < K) out[k] = a;
      else *nrm = a;
    }
  }
}
template <int K, bool NORM>
__global__ void __launch_bounds__(RT) k_multidot(const double* __restrict__ V, long long ldv,
                                                 const double* __restrict__ w, long long N,
                                                 double* __restrict__ partials, unsigned int* counter,
                                                 double* __restrict__ out, const int* __restrict__ skip,
                                                 double* __restrict__ nrm) {
  pdl_entry();
  multidot_body<K, NORM>(V, ldv, w, N, partials, counter, out, skip, nrm);
}

template <int K>
__device__ __forceinline__ void update_multidot_body(const double* __restrict__ V, long long ldv,
                                                     const double* __restrict__ hin, double* __restrict__ w,
                                                     long long N, double* __restrict__ partials,
                                                     unsigned int* counter, double* __restrict__ out) {
  __shared__ double hs[K];
  if (threadIdx.x < K) hs[threadIdx.x] = hin[threadIdx.x];
  __syncthreads();
  double acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = 0.0;
  for (long long e = blockIdx.x * (long long)RT + threadIdx.x; e < N; e += (long long)gridDim.x * RT) {
    double vals[K];
#pragma unroll
    for (int k = 0; k < K; ++k) vals[k] = V[k * ldv + e];
    double we = w[e];
#pragma unroll
    for (int k = 0; k < K; ++k) we = fma(-hs[k], vals[k], we);
    w[e] = we;
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = fma(vals[k], we, acc[k]);
  }
  block_partials<K>(acc, K, partials);
  if (last_block(counter)) final_sums(partials, K, out);
}
template <int K>
__global__ void __launch_bounds__(RT) k_update_multidot(const double* __restrict__ V, long long ldv,
                                                        const double* __restrict__ hin, double* __restrict__ w,
                                                        long long N, double* __restrict__ partials,
                                                        unsigned int* counter, double* __restrict__ out) {
  pdl_entry();
  update_multidot_body<K>(V, ldv, hin, w, N, partials, counter, out);
}

// Column j of H from h1 (+ h2 when `two`), eta = sqrt(s); Givens rotations
// and the residual estimate.  One thread.
__device__ void arnoldi_column(KrylovState* ks, int j, double s, bool two) {
  const int ld = KRYLOV_MAX + 1;
  double* Hj = ks->H + (long long)ld * j;
  for (int i = 0; i <= j; ++i) Hj[i] = two ? ks->h1[i] + ks->h2[i] : ks->h1[i];
  const double eta = sqrt(s);
  Hj[j + 1] = eta;
  ks->eta = eta;
  ks->inv_eta = eta > 0.0 ? 1.0 / eta : 0.0;
  for (int i = 0; i < j; ++i) {                       // previous rotations
    const double a = Hj[i], b = Hj[i + 1];
    Hj[i] = ks->cs[i] * a + ks->sn[i] * b;
    Hj[i + 1] = -ks->sn[i] * a + ks->cs[i] * b;
  }
  const double a = Hj[j], b = Hj[j + 1];
  const double r = hypot(a, b);
  const double c = r > 0.0 ? a / r : 1.0, sn = r > 0.0 ? b / r : 0.0;
  ks->cs[j] = c;
  ks->sn[j] = sn;
  Hj[j] = r;
  Hj[j + 1] = 0.0;
  ks->g[j + 1] = -sn * ks->g[j];
  ks->g[j] = c * ks->g[j];
  const double res = fabs(ks->g[j + 1]);
  ks->resid = res;
  ks->nsteps += 1.0;
  // continue while the estimate is above the tolerance, finite, and the basis grew
  ks->go = (res > ks->thresh && eta > 0.0 && isfinite(res)) ? 1.0 : 0.0;
}

// w -= V h2 (h2 = ks->h2[K0..K0+K)), ||w||^2; last block: column j of H
// (h1 + h2), Givens rotations, residual estimate.  Returns at once when
// `skip` is set.
template <int K>
__device__ __forceinline__ void update_norm_givens_body(const double* __restrict__ V, long long ldv,
                                                        double* __restrict__ w, long long N,
                                                        double* __restrict__ partials, unsigned int* counter,
                                                        KrylovState* ks, int j, int K0,
                                                        const int* __restrict__ skip) {
  if (skip && *skip) return;
  __shared__ double hs[K];
  if (threadIdx.x < K) hs[threadIdx.x] = ks->h2[K0 + threadIdx.x];
  __syncthreads();
  double acc[1] = {0.0};
  for (long long e = blockIdx.x * (long long)RT + threadIdx.x; e < N; e += (long long)gridDim.x * RT) {
    double vals[K];
#pragma unroll
    for (int k = 0; k < K; ++k) vals[k] = V[k * ldv + e];
    double we = w[e];
#pragma unroll
    for (int k = 0; k < K; ++k) we = fma(-hs[k], vals[k], we);
    w[e] = we;
    acc[0] = fma(we, we, acc[0]);
  }
  block_partials<1>(acc, 1, partials);
  if (!last_block(counter) || threadIdx.x >= 32) return;
  const double s = warp_sum_partials(partials, 0);
  if (threadIdx.x == 0) {
    if (skip) ks->passes2 += 1;
    arnoldi_column(ks, j, s, true);
  }
}
template <int K>
__global__ void __launch_bounds__(RT) k_update_norm_givens(const double* __restrict__ V, long long ldv,
                                                           double* __restrict__ w, long long N,
                                                           double* __restrict__ partials, unsigned int* counter,
                                                           KrylovState* ks, int j, int K0,
                                                           const int* __restrict__ skip) {
  pdl_entry();
  update_norm_givens_body<K>(V, ldv, w, N, partials, counter, ks, j, K0, skip);
}

// First-pass update w -= V h1 (h1 = ks->h1[K0..K0+K)), ||w||^2; last block:
// the re-orthogonalisation test against ks->nw0.  Without a second pass the
// column is finished here (H(:,j) = h1).
template <int K>
__global__ void __launch_bounds__(RT) k_update_norm_check(const double* __restrict__ V, long long ldv,
                                                          double* __restrict__ w, long long N,
                                                          double* __restrict__ partials, unsigned int* counter,
                                                          KrylovState* ks, int j, int K0, int single) {
  pdl_entry();
  __shared__ double hs[K];
  if (threadIdx.x < K) hs[threadIdx.x] = ks->h1[K0 + threadIdx.x];
  __syncthreads();
  double acc[1] = {0.0};
  for (long long e = blockIdx.x * (long long)RT + threadIdx.x; e < N; e += (long long)gridDim.x * RT) {
    double vals[K];
#pragma unroll
    for (int k = 0; k < K; ++k) vals[k] = V[k * ldv + e];
    double we = w[e];
#pragma unroll
    for (int k = 0; k < K; ++k) we = fma(-hs[k], vals[k], we);
    w[e] = we;
    acc[0] = fma(we, we, acc[0]);
  }
  block_partials<1>(acc, 1, partials);
  if (!last_block(counter) || threadIdx.x >= 32) return;
  const double s = warp_sum_partials(partials, 0);
  if (threadIdx.x == 0) {
    const bool second = !single && !(s >= 0.5 * ks->nw0);   // also taken when s or nw0 is NaN
    ks->skip2 = second ? 0 : 1;
    if (!second) arnoldi_column(ks, j, s, false);
  }
}

template <int K>
__device__ __forceinline__ void update_only_body(const double* __restrict__ V, long long ldv,
                                                 const double* __restrict__ h, double* __restrict__ w, long long N,
                                                 const int* __restrict__ skip) {
  if (skip && *skip) return;
  __shared__ double hs[K];
  if (threadIdx.x < K) hs[threadIdx.x] = h[threadIdx.x];
  __syncthreads();
  for (long long e = blockIdx.x * (long long)RT + threadIdx.x; e < N; e += (long long)gridDim.x * RT) {
    double vals[K];
#pragma unroll
    for (int k = 0; k < K; ++k) vals[k] = V[k * ldv + e];
    double we = w[e];
#pragma unroll
    for (int k = 0; k < K; ++k) we = fma(-hs[k], vals[k], we);
    w[e] = we;
  }
}
template <int K>
__global__ void __launch_bounds__(RT) k_update_only(const double* __restrict__ V, long long ldv,
                                                    const double* __restrict__ h, double* __restrict__ w,
                                                    long long N, const int* __restrict__ skip) {
  pdl_entry();
  update_only_body<K>(V, ldv, h, w, N, skip);
}

// ---- batched forms: problem blockIdx.y of the batch -----------------------
template <int K, bool NORM>
__global__ void __launch_bounds__(RT) k_multidot_b(Batch<KrylovItem> B, int k0) {
  pdl_entry();
  const KrylovItem& a = B.a[blockIdx.y];
  multidot_body<K, NORM>(a.V + k0 * a.ldv, a.ldv, a.w, a.N, a.partials, a.counter,
                         (a.h_out_is_h2 ? a.ks->h2 : a.ks->h1) + k0, (const int*)nullptr,
                         NORM ? &a.ks->nw0 : (double*)nullptr);
}
template <int K>
__global__ void __launch_bounds__(RT) k_update_multidot_b(Batch<KrylovItem> B) {
  pdl_entry();
  const KrylovItem& a = B.a[blockIdx.y];
  update_multidot_body<K>(a.V, a.ldv, a.ks->h1, a.w, a.N, a.partials, a.counter, a.ks->h2);
}
template <int K>
__global__ void __launch_bounds__(RT) k_update_only_b(Batch<KrylovItem> B, int k0, int second) {
  pdl_entry();
  const KrylovItem& a = B.a[blockIdx.y];
  update_only_body<K>(a.V + k0 * a.ldv, a.ldv, (second ? a.ks->h2 : a.ks->h1) + k0, a.w, a.N, (const int*)nullptr);
}
template <int K>
__global__ void __launch_bounds__(RT) k_update_norm_givens_b(Batch<KrylovItem> B, int j, int k0) {
  pdl_entry();
  const KrylovItem& a = B.a[blockIdx.y];
  update_norm_givens_body<K>(a.V + k0 * a.ldv, a.ldv, a.w, a.N, a.partials, a.counter, a.ks, j, k0,
                             (const int*)nullptr);
}
__global__ void __launch_bounds__(RT) k_scale_by_b(Batch<KrylovItem> B) {
  pdl_entry();
  const KrylovItem& a = B.a[blockIdx.y];
  const double f = a.ks->inv_eta;
  for (long long e = blockIdx.x * (long long)RT + threadIdx.x; e < a.N; e += (long long)gridDim.x * RT) a.w[e] *= f;
}

// run F.template operator()<K>() for the runtime K in 1..KC
template <typename F>
static void with_k(int K, F&& f) {
  switch (K) {
#define OK_K(k) case k: f(std::integral_constant<int, k>{}); break;
    OK_K(1) OK_K(2) OK_K(3) OK_K(4) OK_K(5) OK_K(6) OK_K(7) OK_K(8)
    OK_K(9) OK_K(10) OK_K(11) OK_K(12) OK_K(13) OK_K(14) OK_K(15) OK_K(16)
#undef OK_K
    default: break;
  }
}

__global__ void __launch_bounds__(RT) k_sumsq(const double* __restrict__ x, long long N,
                                              double* __restrict__ partials, unsigned int* counter,
                                              double* __restrict__ out) {
  pdl_entry();
  double acc[1] = {0.0};
  for (long long e = blockIdx.x * (long long)RT + threadIdx.x; e < N; e += (long long)gridDim.x * RT)
    acc[0] = fma(x[e], x[e], acc[0]);
  block_partials<1>(acc, 1, partials);
  if (!last_block(counter) || threadIdx.x >= 32) return;
  const double s = warp_sum_partials(partials, 0);
  if (threadIdx.x == 0) *out = sqrt(s);
}

__global__ void __launch_bounds__(RT) k_scale_by(double* __restrict__ w, long long N,
                                                 const double* __restrict__ factor) {
  pdl_entry();
  const double f = *factor;
  for (long long e = blockIdx.x * (long long)RT + threadIdx.x; e < N; e += (long long)gridDim.x * RT) w[e] *= f;
}

__global__ void k_cycle_start(KrylovState* ks, const double* __restrict__ beta, double thresh) {
  pdl_entry();
  if (threadIdx.x == 0) {
    const double b = *beta;
    ks->beta = b;
    ks->inv_beta = b > 0.0 ? 1.0 / b : 0.0;
    for (int i = 0; i <= KRYLOV_MAX; ++i) ks->g[i] = 0.0;
    ks->g[0] = b;
    ks->resid = b;
    ks->go = 1.0;
    ks->nsteps = 0.0;
    ks->thresh = thresh;
  }
}

// First node of a conditional Arnoldi-step graph: the step's body runs only
// while the cycle goes on (the previous step's stop test, on the device).
__global__ void k_cond_set(cudaGraphConditionalHandle h, const KrylovState* __restrict__ ks) {
  cudaGraphSetConditional(h, ks->go != 0.0 ? 1u : 0u);
}
void* cond_set_kernel() { return (void*)k_cond_set; }

// back substitution R y = g, R = rotated H (k x k upper triangular)
__global__ void k_lsq(KrylovState* ks, int k) {
  pdl_entry();
  if (threadIdx.x == 0) {
    const int ld = KRYLOV_MAX + 1;
    for (int i = k - 1; i >= 0; --i) {
      double s = ks->g[i];
      for (int c = i + 1; c < k; ++c) s -= ks->H[i + ld * c] * ks->y[c];
      const double d = ks->H[i + ld * i];
      ks->y[i] = d != 0.0 ? s / d : 0.0;
    }
  }
}

template <typename TZ>
__global__ void __launch_bounds__(RT) k_multi_axpy(const TZ* __restrict__ Z, long long ldz, int K,
                                                   const KrylovState* __restrict__ ks, double* __restrict__ x,
                                                   long long N) {
  pdl_entry();
  __shared__ double ys[KRYLOV_MAX];
  if (threadIdx.x < KRYLOV_MAX) ys[threadIdx.x] = threadIdx.x < K ? ks->y[threadIdx.x] : 0.0;
  __syncthreads();
  for (long long e = blockIdx.x * (long long)RT + threadIdx.x; e < N; e += (long long)gridDim.x * RT) {
    double acc = x[e];
    for (int k = 0; k < K; ++k) {
      double zk;
      if constexpr (std::is_same<TZ, float>::value) zk = f2d_exact(Z[k * ldz + e]);
      else if constexpr (std::is_same<TZ, __half>::value) zk = f2d_exact(__half2float(Z[k * ldz + e]));
      else zk = Z[k * ldz + e];
      acc = fma(ys[k], zk, acc);
    }
    x[e] = acc;
  }
}

template <typename TX, typename TY>
__global__ void __launch_bounds__(RT) k_axpby(long long N, double a, const TX* __restrict__ x, double b,
                                              TY* __restrict__ y) {
  pdl_entry();
  for (long long e = blockIdx.x * (long long)RT + threadIdx.x; e < N; e += (long long)gridDim.x * RT) {
    double v = a * (double)x[e];
    if constexpr (std::is_same<TY, __half>::value) {
      if (b != 0.0) v = fma(b, (double)__half2float(y[e]), v);
      y[e] = __float2half_rn((float)v);
    } else {
      if (b != 0.0) v = fma(b, (double)y[e], v);
      y[e] = (TY)v;
    }
  }
}

__global__ void __launch_bounds__(RT) k_check_finite(const double* __restrict__ x, long long N, int* flag) {
  pdl_entry();
  int bad = 0;
  for (long long e = blockIdx.x * (long long)RT + threadIdx.x; e < N; e += (long long)gridDim.x * RT)
    bad |= !isfinite(x[e]);
  bad = __syncthreads_or(bad);
  if (bad && threadIdx.x == 0) atomicOr(flag, 1);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
// out[0..K) = V^T w (chunks of KC vectors); with nw0, also ||w||^2 there (first chunk)
void launch_multidot(const double* V, long long ldv, int K, const double* w, long long N, RedScratch rs,
                     double* out, cudaStream_t s, const int* skip, double* nw0) {
  for (int k0 = 0; k0 < K; k0 += KC) {
    const int kk = K - k0 < KC ? K - k0 : KC;
    with_k(kk, [&](auto KK) {
      constexpr int KV = decltype(KK)::value;
      if (k0 == 0 && nw0)
        launch_k(k_multidot<KV, true>, krylov_blocks(), RT, 0, s, V + k0 * ldv, ldv, w, N, rs.partials,
                 rs.counter, out + k0, skip, nw0);
      else
        launch_k(k_multidot<KV, false>, krylov_blocks(), RT, 0, s, V + k0 * ldv, ldv, w, N, rs.partials,
                 rs.counter, out + k0, skip, (double*)nullptr);
    });
  }
}

void launch_update_multidot(const double* V, long long ldv, int K, const double* h_in, double* w, long long N,
                            RedScratch rs, double* h_out, cudaStream_t s) {
  if (K <= KC) {
    with_k(K, [&](auto KK) {
      launch_k(k_update_multidot<decltype(KK)::value>, krylov_blocks(), RT, 0, s, 
                          V, ldv, h_in, w, N, rs.partials, rs.counter, h_out);
    });
    return;
  }
  for (int k0 = 0; k0 < K; k0 += KC) {   // all updates first, then the dots of the final w
    const int kk = K - k0 < KC ? K - k0 : KC;
    with_k(kk, [&](auto KK) {
      launch_k(k_update_only<decltype(KK)::value>, krylov_blocks(), RT, 0, s, V + k0 * ldv, ldv, h_in + k0,
                                                                                       w, N, (const int*)nullptr);
    });
  }
  launch_multidot(V, ldv, K, w, N, rs, h_out, s, nullptr, nullptr);
}

void launch_update_norm_givens(const double* V, long long ldv, int K, double* w, long long N, RedScratch rs,
                               KrylovState* ks, int j, cudaStream_t s, const int* skip) {
  int k0 = 0;
  for (; K - k0 > KC; k0 += KC) {
    // h2 lives in device memory inside ks; chunk offsets index it directly
    launch_k(k_update_only<KC>, krylov_blocks(), RT, 0, s, V + k0 * ldv, ldv, ks->h2 + k0, w, N, skip);
  }
  with_k(K - k0, [&](auto KK) {
    launch_k(k_update_norm_givens<decltype(KK)::value>, krylov_blocks(), RT, 0, s, 
                        V + k0 * ldv, ldv, w, N, rs.partials, rs.counter, ks, j, k0, skip);
  });
}

void launch_update_norm_check(const double* V, long long ldv, int K, double* w, long long N, RedScratch rs,
                              KrylovState* ks, int j, cudaStream_t s, bool single) {
  int k0 = 0;
  for (; K - k0 > KC; k0 += KC)
    launch_k(k_update_only<KC>, krylov_blocks(), RT, 0, s, V + k0 * ldv, ldv, ks->h1 + k0, w, N,
             (const int*)nullptr);
  with_k(K - k0, [&](auto KK) {
    launch_k(k_update_norm_check<decltype(KK)::value>, krylov_blocks(), RT, 0, s, V + k0 * ldv, ldv, w, N,
             rs.partials, rs.counter, ks, j, k0, single ? 1 : 0);
  });
}

void launch_scale_by(double* w, long long N, const double* factor, cudaStream_t s) {
  launch_k(k_scale_by, krylov_blocks(), RT, 0, s, w, N, factor);
}

void launch_norm(const double* x, long long N, RedScratch rs, double* out, cudaStream_t s) {
  launch_k(k_sumsq, krylov_blocks(), RT, 0, s, x, N, rs.partials, rs.counter, out);
}

void launch_cycle_start(KrylovState* ks, const double* beta, double thresh, cudaStream_t s) {
  launch_k(k_cycle_start, 1, 32, 0, s, ks, beta, thresh);
}

void launch_lsq(KrylovState* ks, int k, cudaStream_t s) { launch_k(k_lsq, 1, 32, 0, s, ks, k); }

template <typename TZ>
void launch_multi_axpy(const TZ* Z, long long ldz, int K, const KrylovState* ks, double* x, long long N,
                       cudaStream_t s) {
  launch_k(k_multi_axpy<TZ>, krylov_blocks(), RT, 0, s, Z, ldz, K, ks, x, N);
}
template void launch_multi_axpy<double>(const double*, long long, int, const KrylovState*, double*, long long,
                                        cudaStream_t);
template void launch_multi_axpy<float>(const float*, long long, int, const KrylovState*, double*, long long,
                                       cudaStream_t);
template void launch_multi_axpy<__half>(const __half*, long long, int, const KrylovState*, double*, long long,
                                        cudaStream_t);

template <typename TX, typename TY>
void launch_axpby(long long N, double a, const TX* x, double b, TY* y, cudaStream_t s) {
  launch_k(k_axpby<TX, TY>, krylov_blocks(), RT, 0, s, N, a, x, b, y);
}
template void launch_axpby<double, double>(long long, double, const double*, double, double*, cudaStream_t);
template void launch_axpby<float, double>(long long, double, const float*, double, double*, cudaStream_t);
template void launch_axpby<double, float>(long long, double, const double*, double, float*, cudaStream_t);
template void launch_axpby<float, float>(long long, double, const float*, double, float*, cudaStream_t);
template void launch_axpby<float, __half>(long long, double, const float*, double, __half*, cudaStream_t);

void launch_check_finite(const double* x, long long N, int* flag, cudaStream_t s) {
  launch_k(k_check_finite, krylov_blocks(), RT, 0, s, x, N, flag);
}

// One CGS2 Arnoldi orthogonalisation (h1 = V^T w; w -= V h1, h2 = V^T w;
// w -= V h2, column j, Givens; w /= eta) of `count` problems per launch, the
// same kernels' arithmetic as launch_multidot / launch_update_multidot /
// launch_update_norm_givens / launch_scale_by.  K = j + 1 basis vectors.
void launch_cgs2_batch(const KrylovItem* items, int count, int K, int j, cudaStream_t s) {
  Batch<KrylovItem> B;
  for (int i = 0; i < count; ++i) B.a[i] = items[i];
  const dim3 grid(krylov_blocks(), count);
  for (int k0 = 0; k0 < K; k0 += KC) {                    // h1
    const int kk = K - k0 < KC ? K - k0 : KC;
    with_k(kk, [&](auto KK) { launch_k(k_multidot_b<decltype(KK)::value, false>, grid, RT, 0, s, B, k0); });
  }
  if (K <= KC) {                                          // w -= V h1, h2 = V^T w
    with_k(K, [&](auto KK) { launch_k(k_update_multidot_b<decltype(KK)::value>, grid, RT, 0, s, B); });
  } else {
    for (int k0 = 0; k0 < K; k0 += KC) {
      const int kk = K - k0 < KC ? K - k0 : KC;
      with_k(kk, [&](auto KK) { launch_k(k_update_only_b<decltype(KK)::value>, grid, RT, 0, s, B, k0, 0); });
    }
    Batch<KrylovItem> B2 = B;                             // h2 = V^T w into h2: multidot writes h1 + k0
    for (int i = 0; i < count; ++i) B2.a[i].h_out_is_h2 = 1;
    for (int k0 = 0; k0 < K; k0 += KC) {
      const int kk = K - k0 < KC ? K - k0 : KC;
      with_k(kk, [&](auto KK) { launch_k(k_multidot_b<decltype(KK)::value, false>, grid, RT, 0, s, B2, k0); });
    }
  }
  int k0 = 0;                                             // w -= V h2, ||w||, column j
  for (; K - k0 > KC; k0 += KC) launch_k(k_update_only_b<KC>, grid, RT, 0, s, B, k0, 1);
  with_k(K - k0, [&](auto KK) { launch_k(k_update_norm_givens_b<decltype(KK)::value>, grid, RT, 0, s, B, j, k0); });
  launch_k(k_scale_by_b, grid, RT, 0, s, B);
}

}  // namespace okg
