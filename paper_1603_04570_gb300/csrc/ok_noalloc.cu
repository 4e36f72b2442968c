// ok_noalloc.cu -- y = J(u_k) z without any device allocation.
//
// ok_apply_jacobian needs a handle from ok_grid_create, which allocates the
// coefficient store of C = -eps^2 K - M_E(u_k) (and everything else the solver
// uses) with cudaMalloc.  Some callers cannot allocate: applications that own
// all device memory through their own allocator or run under a fixed memory
// budget, and latency-critical loops where cudaMalloc's implicit device-wide
// synchronisation is not acceptable.  This file gives them one entry point
// that runs the same two kernels (coefficient assembly, then the Jacobian
// apply) with the coefficient store in a file-scope static device array.
//
// Limits and sharing:
//   * the static store holds (1 + NPOS) float64 + (1 + NPOS) float32 values
//     per vertex in OKNA_SCRATCH_BYTES = 16 MiB: N_v <= 349,525 in 2D
//     (n <= 590) and N_v <= 174,762 in 3D (n <= 54); larger grids are rejected;
//   * the array lives on every GPU that loads the library until the process
//     exits;
//   * every call uses the same array and leaves the last call's coefficients
//     in it: calls whose work overlaps on the GPU (two streams, two threads)
//     race; serialise them;
//   * the first call on a device looks up the array's device address
//     (cudaGetSymbolAddress) and uploads the stencil tables; make that first
//     call before any stream capture.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/ok.h"
#include "ok_internal.cuh"
#include "ok_kernels.h"

using namespace okg;

namespace {

constexpr size_t OKNA_SCRATCH_BYTES = 16u << 20;
constexpr int OKNA_MAX_DEVICES = 64;
constexpr int OKNA_TAB = 27 * 15;   // largest class table (3D)

// Coefficient store: float64 part first, float32 copy after it.
static __device__ __align__(256) unsigned char g_okna_scratch[OKNA_SCRATCH_BYTES];
// Reference (h = 1) stencil tables of M and K for dim 2 and dim 3.
static __device__ __align__(256) double g_okna_tables[4 * OKNA_TAB];

struct DeviceSetup {
  bool ready = false;
  unsigned char* scratch = nullptr;
  double* tables = nullptr;
};
DeviceSetup g_setup[OKNA_MAX_DEVICES];
std::mutex g_setup_mutex;
int na_fail(int status, const std::string& msg) {
  okg::set_last_error(msg.c_str());   // reported by ok_last_error()
  return status;
}

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// once per device, with that device current
int setup_device(int dev, DeviceSetup** out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  DeviceSetup& s = g_setup[dev];
  if (!s.ready) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_okna_scratch);
    if (e != cudaSuccess) return na_fail(OK_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    s.scratch = (unsigned char*)p;
    e = cudaGetSymbolAddress(&p, g_okna_tables);
    if (e != cudaSuccess) return na_fail(OK_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    s.tables = (double*)p;
    double host[4 * OKNA_TAB];
    std::memset(host, 0, sizeof(host));
    reference_tables(2, host + 0 * OKNA_TAB, host + 1 * OKNA_TAB);
    reference_tables(3, host + 2 * OKNA_TAB, host + 3 * OKNA_TAB);
    e = cudaMemcpy(s.tables, host, sizeof(host), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return na_fail(OK_ERR_CUDA, std::string("table upload: ") + cudaGetErrorString(e));
    s.ready = true;
  }
  *out = &s;
  return OK_SUCCESS;
}

}  // namespace

extern "C" int ok_apply_jacobian_noalloc(int dim, int n, const ok_params* p, const double* u_k, const double* z,
                                         double* y, ok_stream stream) {
  if (dim != 2 && dim != 3) return na_fail(OK_ERR_INVALID_ARG, "dim must be 2 or 3");
  if (n < 2) return na_fail(OK_ERR_INVALID_ARG, "n must be >= 2");
  if (!p || !u_k || !z || !y) return na_fail(OK_ERR_INVALID_ARG, "NULL argument");
  if (!(p->eps > 0) || !(p->dt > 0) || !(p->theta > 0 && p->theta <= 1) || !(p->sigma >= 0))
    return na_fail(OK_ERR_INVALID_ARG, "params out of range (need eps > 0, dt > 0, 0 < theta <= 1, sigma >= 0)");
  const int nslot = dim == 2 ? Topo<2>::NSLOT : Topo<3>::NSLOT;
  const double nvd = std::pow((double)(n + 1), dim);
  const double need = nvd * nslot * (sizeof(double) + sizeof(float));
  if (need > (double)OKNA_SCRATCH_BYTES)
    return na_fail(OK_ERR_INVALID_ARG,
                   "grid too large for the static coefficient store: needs " + std::to_string((long long)need) +
                       " bytes, the store holds " + std::to_string(OKNA_SCRATCH_BYTES) +
                       " (2D: n <= 590, 3D: n <= 54); use ok_grid_create + ok_apply_jacobian");
  if (!on_device(u_k) || !on_device(z) || !on_device(y))
    return na_fail(OK_ERR_INVALID_ARG, "u_k, z and y must be device arrays (host arrays would need staging memory)");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return na_fail(OK_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= OKNA_MAX_DEVICES) return na_fail(OK_ERR_INVALID_ARG, "device index out of range");
  DeviceSetup* s = nullptr;
  int st = setup_device(dev, &s);
  if (st != OK_SUCCESS) return st;

  const Geom g = make_geom(dim, n);
  const double h = 1.0 / n;
  ResidualCoefs rc;
  std::memset(&rc, 0, sizeof(rc));
  rc.hd = std::pow(h, dim);
  rc.hk = std::pow(h, dim - 2);
  rc.eps2 = p->eps * p->eps;
  rc.vol = rc.hd / (dim == 2 ? 2.0 : 6.0);
  rc.a4 = dim == 2 ? 2.0 / 720.0 : 6.0 / 5040.0;
  rc.a2 = dim == 2 ? 2.0 / 24.0 : 6.0 / 120.0;
  JCoefs jc;
  jc.a11hd = (1.0 + p->dt * p->theta * p->sigma) * rc.hd;
  jc.dthhk = p->dt * p->theta * rc.hk;
  jc.hd = rc.hd;
  jc.alpha = 1.0;
  jc.beta = 0.0;

  double* coef = (double*)s->scratch;
  float* coef32 = (float*)(s->scratch + (size_t)nslot * g.nv * sizeof(double));
  const double* WM = s->tables + (dim == 2 ? 0 : 2) * OKNA_TAB;
  const double* WK = s->tables + (dim == 2 ? 1 : 3) * OKNA_TAB;
  cudaStream_t cs = (cudaStream_t)stream;
  // every coefficient slot is rewritten by the assembly kernel, so nothing
  // from the previous call needs clearing
  launch_assemble_c(dim, g, rc, u_k, coef, coef32, cs);
  launch_apply_j<double>(dim, g, WM, WK, jc, coef, z, y, nullptr, cs);
  e = cudaGetLastError();
  if (e != cudaSuccess) return na_fail(OK_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  okg::set_last_error("");
  return OK_SUCCESS;
}
