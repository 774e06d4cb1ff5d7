// Allocation-free CFL step: a variant of the CFL reduction for callers that
// cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is not allowed or not
// wanted -- inside a host callback or a custom allocator hook, in a process
// whose device memory is owned entirely by another framework's caching
// allocator, or under a memory budget that forbids growth after start-up.
// Such callers still own the state (inputs) and the dt slot (output); the
// only memory this entry point needs besides those is its reduction
// scratch, which lives in the file-scope device array below.
//
// The scratch is a static __device__ array: every GPU that loads this
// library's device code holds it (about 2 MiB) until the process exits.
// With the runtime's default lazy module loading, the device code (and the
// array) is loaded at the first kernel launch or symbol lookup on that
// device, so the first call may need device memory; later calls need none.
// The address cache is per device ordinal and assumes the device's primary
// context.  All calls share the array, so calls whose work overlaps on the
// GPU (different streams, or different host threads) race on it; serialise
// them.
#include <mutex>

#include "runtime.hpp"

namespace aeth {
namespace {

// One partial minimum per x-row (ny * nz rows) plus the status word.
constexpr int kNoAllocMaxRows = 1 << 18;

struct NoAllocScratch {
  double partial[kNoAllocMaxRows];
  int status;
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// Device address of g_noalloc_scratch per device, looked up once per device.
std::mutex g_noalloc_mu;
constexpr int kMaxDevices = 64;
void* g_noalloc_ptr[kMaxDevices] = {nullptr};

__device__ __forceinline__ double warp_min_na(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Eq. 11 on the plain FP64 layout of the C ABI: one warp per x-row writes
// that row's minimum of dx_d / (|v_d| + c_f,d) (eight rows per CUDA block,
// so short rows do not leave most of a block idle).
constexpr int kRowsPerBlock = 8;

__global__ void __launch_bounds__(32 * kRowsPerBlock)
    k_dt_rows_plain(const double* __restrict__ cons, const double* __restrict__ b1,
                    const double* __restrict__ b2, const double* __restrict__ b3, int nx, int ny,
                    int nz, double dx1, double dx2, double dx3, double gamma, double rho_floor,
                    double p_floor, int mhd, NoAllocScratch* s) {
  const int r = blockIdx.x * kRowsPerBlock + (int)(threadIdx.x >> 5);
  const int lane = (int)threadIdx.x & 31;
  if (r >= ny * nz) return;   // whole warps leave together
  const int j = r % ny, k = r / ny;
  const long long nc = (long long)nx * ny * nz;
  const double w[3] = {dx1, dx2, dx3};
  double m = INFINITY;
  bool bad = false;
  for (int i = lane; i < nx; i += 32) {
    const long long c = ((long long)k * ny + j) * nx + i;
    double rho = cons[c];
    if (!(rho >= rho_floor)) { if (!(rho == rho)) bad = true; rho = rho_floor; }
    const double v[3] = {cons[nc + c] / rho, cons[2 * nc + c] / rho, cons[3 * nc + c] / rho};
    double bc[3] = {0, 0, 0};
    if (mhd) {
      bc[0] = 0.5 * (b1[((long long)k * ny + j) * (nx + 1) + i] +
                     b1[((long long)k * ny + j) * (nx + 1) + i + 1]);
      bc[1] = 0.5 * (b2[((long long)k * (ny + 1) + j) * nx + i] +
                     b2[((long long)k * (ny + 1) + j + 1) * nx + i]);
      bc[2] = 0.5 * (b3[((long long)k * ny + j) * nx + i] +
                     b3[((long long)(k + 1) * ny + j) * nx + i]);
    }
    double pr = (gamma - 1.0) * (cons[4 * nc + c] - 0.5 * rho * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) -
                                 0.5 * (bc[0] * bc[0] + bc[1] * bc[1] + bc[2] * bc[2]));
    if (!(pr >= p_floor)) { if (!(pr == pr)) bad = true; pr = p_floor; }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double cf = fast_speed(gamma, rho, pr, bc[d], bc[(d + 1) % 3], bc[(d + 2) % 3]);
      const double dtd = w[d] / (fabs(v[d]) + cf);
      if (!(dtd > 0.0)) bad = true;
      m = fmin(m, dtd);
    }
  }
  m = warp_min_na(m);
  if (lane == 0) s->partial[r] = m;
  if (bad) atomicOr(&s->status, 1);
}

__global__ void k_dt_rows_final(const NoAllocScratch* __restrict__ s, int rows, double scale,
                                double* __restrict__ dt) {
  __shared__ double sm[32];
  double m = INFINITY;
  for (int t = threadIdx.x; t < rows; t += blockDim.x) m = fmin(m, s->partial[t]);
  m = warp_min_na(m);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : INFINITY;
    v = warp_min_na(v);
    // a non-finite state gives a NaN step, never a silently finite one
    if (threadIdx.x == 0) *dt = s->status ? NAN : scale * v;
  }
}

}  // namespace
}  // namespace aeth

extern "C" aeth_status aeth_cfl_dt_noalloc(const double* d_cons, const double* d_b1,
                                           const double* d_b2, const double* d_b3, int nx,
                                           int ny, int nz, double dx1, double dx2, double dx3,
                                           double gamma, double rho_floor, double p_floor,
                                           double cfl, int mhd, double* d_dt,
                                           void* cuda_stream) {
  using namespace aeth;
  if (!d_cons || !d_dt || (mhd && (!d_b1 || !d_b2 || !d_b3))) return AETH_ERR_ARG;
  if (nx < 1 || ny < 1 || nz < 1) return AETH_ERR_ARG;
  if (!(dx1 > 0 && dx2 > 0 && dx3 > 0 && gamma > 1.0 && cfl > 0.0 && cfl <= 1.0))
    return AETH_ERR_ARG;
  const long long rows = (long long)ny * nz;
  if (rows > kNoAllocMaxRows) return AETH_ERR_ARG;   // ny * nz beyond the scratch
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return AETH_ERR_CUDA;
  void* ptr = nullptr;
  {
    // set-up, once per device, with that device current
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess) return AETH_ERR_CUDA;
      g_noalloc_ptr[dev] = ptr;
    }
    ptr = g_noalloc_ptr[dev];
  }
  NoAllocScratch* s = static_cast<NoAllocScratch*>(ptr);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // the status word must start at zero; the partials are all rewritten
  if (cudaMemsetAsync(&s->status, 0, sizeof(int), st) != cudaSuccess) return AETH_ERR_CUDA;
  k_dt_rows_plain<<<(unsigned)((rows + kRowsPerBlock - 1) / kRowsPerBlock), 32 * kRowsPerBlock, 0,
                    st>>>(d_cons, d_b1, d_b2, d_b3, nx, ny, nz, dx1, dx2, dx3, gamma, rho_floor,
                          p_floor, mhd, s);
  k_dt_rows_final<<<1, 1024, 0, st>>>(s, (int)rows, cfl, d_dt);
  if (cudaGetLastError() != cudaSuccess) return AETH_ERR_CUDA;
  return AETH_OK;
}
