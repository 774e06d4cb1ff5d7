// Learned Riemann flux: a 14 -> 128 -> 128 -> 128 -> 7 MLP (SiLU hidden
// layers) that replaces the HLLD solve of Sec. 2.4 face by face, with a
// per-face residual check against HLLE and a positivity check of the
// implied intermediate states; failing faces fall back to exact HLLD.  The
// paper has no learned flux: this is the learned-flux configuration of the
// benchmark set.
//
// Inputs are made dimensionless with the left density rho_L and the
// reference speed c = max(c_f,L, c_f,R) (ideal MHD is invariant under that
// scaling), which drops rho_L = 1 and leaves 14 inputs, padded to 16 for the
// tensor-core k-step.  Outputs (7 fluxes) are scaled back by rho_L c,
// rho_L c^2, rho_L c^3 gamma/(gamma-1) and sqrt(rho_L) c^2.  A face is
// accepted if every flux lies within mlp_tau of the HLL dissipation bracket
// around HLLE plus 2e-2 of its scale.
//
// Training runs on the GPU with the project's own FP32 kernels (tiled SGEMM,
// SiLU backward, Adam).  Inference runs on the tensor cores in BF16 with
// FP32 accumulation (mma.sync m16n8k16): a warp pushes 16 faces at a time
// through all four layers, keeping the hidden activations in registers
// (each layer's accumulator fragments are exactly the next layer's A
// fragments), with the BF16 weights staged once per CTA in shared memory.
#include <cstring>
#include <vector>

#include <cuda_bf16.h>

#include "runtime.hpp"
#include "stage.cuh"
#include "mlp_face.cuh"

namespace aeth {

template <typename R>
void launch_fill(const BlockPtrs<R>& P, R* const* arrs, int nv, cudaStream_t st);

constexpr int MLP_IN = 14, MLP_H = 128, MLP_OUT = 7;
constexpr int MLP_INP = 16, MLP_OUTP = 8;   // padded widths
constexpr long long MLP_NPARAM = (long long)MLP_H * MLP_IN + MLP_H + 2LL * (MLP_H * MLP_H + MLP_H) +
                                 (long long)MLP_OUT * MLP_H + MLP_OUT;

// ------------------------------------------------------------------------
// training samples: PLM face states of the solver's current state, HLLD
// flux targets, both dimensionless
// ------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256)
    k_mlp_samples(BlockPtrs<R> P, int stride, long long capacity, float* __restrict__ X,
                  float* __restrict__ Y, unsigned long long* count, R gamma, R rho_floor,
                  R p_floor, int mhd) {
  const Layout L = P.L;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z * blockDim.z + threadIdx.z;
  if (i >= L.n[0] || j >= L.n[1] || k >= L.n[2]) return;
  const long long lin = ((long long)k * L.n[1] + j) * L.n[0] + i;
  if (lin % stride != 0) return;
  const R* ub = P.reg[0][0];
  const long long pitch = P.pitch;
  const R gm1 = gamma - R(1);
#pragma unroll 1
  for (int d = 0; d < 3; ++d) {
    const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    const int slot[7] = {0, 1 + d, 1 + t1, 1 + t2, 4, 5 + t1, 5 + t2};
    R st[4][8];
    for (int t = 0; t < 4; ++t) {   // PLM stencil cells f-2 .. f+1
      int c3[3] = {i, j, k};
      c3[d] += t - 2;
      R w[8];
      if (mhd) prim_cell_s<R, false, true>(L, ub, pitch, L.idx(c3[0], c3[1], c3[2]), gm1, rho_floor, p_floor, w);
      else prim_cell_s<R, false, false>(L, ub, pitch, L.idx(c3[0], c3[1], c3[2]), gm1, rho_floor, p_floor, w);
      for (int v = 0; v < 8; ++v) st[t][v] = w[v];
    }
    R wl[7], wr[7];
    for (int v = 0; v < 7; ++v) {
      const int q = slot[v];
      wl[v] = st[1][q] + R(0.5) * vl_slope(st[0][q], st[1][q], st[2][q]);
      wr[v] = st[2][q] - R(0.5) * vl_slope(st[1][q], st[2][q], st[3][q]);
    }
    const R bn = mhd ? ub[(5 + d) * pitch + L.idx(i, j, k)] : R(0);
    if (!mhd) { wl[5] = wl[6] = wr[5] = wr[6] = R(0); }
    float x[16], sc[7], y[7];
    const FaceScale s = mlp_features(wl, wr, bn, gamma, x);
    mlp_scale_out(s, (float)gamma, sc);
    {
      // targets in FP64: F_HLLD - F_HLLE cancels for small jumps
      double dl[7], dr[7], fx[7];
      for (int q = 0; q < 7; ++q) { dl[q] = (double)wl[q]; dr[q] = (double)wr[q]; }
      hlld((double)gamma, dl, dr, (double)bn, fx);
      mlp_target((double)gamma, dl, dr, (double)bn, fx, sc, y);
    }
    const unsigned long long slot_id = atomicAdd(count, 1ull);
    if ((long long)slot_id >= capacity) continue;
    for (int q = 0; q < 16; ++q) X[slot_id * 16 + q] = x[q];
    for (int q = 0; q < 7; ++q) Y[slot_id * 8 + q] = y[q];
    Y[slot_id * 8 + 7] = 0.0f;
  }
}

// ------------------------------------------------------------------------
// FP32 training kernels
// ------------------------------------------------------------------------
// C[m][n] = alpha * sum_k A(m,k) B(k,n) + beta * C[m][n]; A(m,k) = A[m*sam + k*sak],
// B(k,n) = B[k*sbk + n*sbn], C row-major with ldc.  64x64 tiles, 256 threads.
__global__ void __launch_bounds__(256)
    k_sgemm(int M, int N, int K, float alpha, const float* __restrict__ A, long long sam,
            long long sak, const float* __restrict__ B, long long sbk, long long sbn, float beta,
            float* __restrict__ C, long long ldc) {
  __shared__ float As[16][64 + 4];
  __shared__ float Bs[16][64 + 4];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int e = threadIdx.x; e < 16 * 64; e += 256) {
      const int kk = e / 64, mm = e % 64;
      const int gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < M && gk < K) ? A[gm * sam + gk * sak] : 0.0f;
      const int gn = n0 + mm;
      Bs[kk][mm] = (gn < N && gk < K) ? B[gk * sbk + gn * sbn] : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) { a[q] = As[kk][ty * 4 + q]; b[q] = Bs[kk][tx * 4 + q]; }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] += a[p] * b[q];
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int gm = m0 + ty * 4 + p, gn = n0 + tx * 4 + q;
      if (gm < M && gn < N) {
        float v = alpha * acc[p][q];
        if (beta != 0.0f) v += beta * C[gm * ldc + gn];
        C[gm * ldc + gn] = v;
      }
    }
}

__device__ __forceinline__ float silu_f(float z) { return z / (1.0f + __expf(-z)); }
__device__ __forceinline__ float dsilu_f(float z) {
  const float s = 1.0f / (1.0f + __expf(-z));
  return s * (1.0f + z * (1.0f - s));
}

// Z[s][o] += b[o]; A = silu(Z) (or A = Z for the output layer)
__global__ void k_bias_act(float* __restrict__ Z, float* __restrict__ Aout, const float* __restrict__ b,
                           int n, int width, int ld, int act) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n * width) return;
  const int s = (int)(t / width), o = (int)(t % width);
  const float z = Z[(long long)s * ld + o] + b[o];
  Z[(long long)s * ld + o] = z;
  Aout[(long long)s * ld + o] = act ? silu_f(z) : z;
}

// dY = (Yhat - Y) / n over the 7 real outputs; loss partial sums
__global__ void k_loss(const float* __restrict__ Yh, const float* __restrict__ Y, float* __restrict__ dY,
                       int n, float* __restrict__ loss) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.0f;
  if (s < n) {
    for (int o = 0; o < MLP_OUT; ++o) {
      const float e = Yh[(long long)s * MLP_OUTP + o] - Y[(long long)s * MLP_OUTP + o];
      dY[(long long)s * MLP_OUTP + o] = e / n;
      l += 0.5f * e * e;
    }
    dY[(long long)s * MLP_OUTP + 7] = 0.0f;
  }
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, l / n);
}

// db[o] = sum_s dZ[s][o]
__global__ void k_colsum(const float* __restrict__ dZ, float* __restrict__ db, int n, int width, int ld) {
  const int o = blockIdx.x;
  float acc = 0.0f;
  for (int s = threadIdx.x; s < n; s += blockDim.x) acc += dZ[(long long)s * ld + o];
  for (int q = 16; q > 0; q >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, q);
  __shared__ float sm[32];
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    float v = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : 0.0f;
    for (int q = 16; q > 0; q >>= 1) v += __shfl_xor_sync(0xffffffffu, v, q);
    if (threadIdx.x == 0) db[o] = v;
  }
}

// dZ = dA * silu'(Z)
__global__ void k_dsilu(float* __restrict__ dA, const float* __restrict__ Z, long long n) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) dA[t] *= dsilu_f(Z[t]);
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, long long n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const float gt = g[t];
  const float mt = b1 * m[t] + (1.0f - b1) * gt;
  const float vt = b2 * v[t] + (1.0f - b2) * gt * gt;
  m[t] = mt;
  v[t] = vt;
  p[t] -= lr * (mt / c1) / (sqrtf(vt / c2) + eps);
}

static void sgemm(cudaStream_t st, int M, int N, int K, float alpha, const float* A, long long sam,
                  long long sak, const float* B, long long sbk, long long sbn, float beta, float* C,
                  long long ldc) {
  dim3 grd((N + 63) / 64, (M + 63) / 64);
  k_sgemm<<<grd, 256, 0, st>>>(M, N, K, alpha, A, sam, sak, B, sbk, sbn, beta, C, ldc);
}

// Parameter offsets of the unpadded layout (per layer: W[out][in], b[out]).
static void layer_offsets(long long* off) {
  const int dims[5] = {MLP_IN, MLP_H, MLP_H, MLP_H, MLP_OUT};
  off[0] = 0;
  for (int l = 0; l < 4; ++l) off[l + 1] = off[l] + (long long)dims[l + 1] * dims[l] + dims[l + 1];
}

}  // namespace aeth

using namespace aeth;

extern "C" aeth_status aeth_mlp_work_floats(int n, size_t* out) {
  if (n <= 0 || !out) return AETH_ERR_ARG;
  // Z1..Z3, A1..A3 (n x 128 each), Yhat (n x 8), dY (n x 8), two dZ buffers
  *out = (size_t)n * (6 * MLP_H + 2 * MLP_OUTP + 2 * MLP_H);
  return AETH_OK;
}

extern "C" aeth_status aeth_mlp_grad(const float* d_params, const float* d_X, const float* d_Y,
                                     int n, float* d_grad, float* d_work, size_t work_floats,
                                     float* d_loss, void* cuda_stream) {
  if (!d_params || !d_X || !d_Y || !d_grad || !d_work || !d_loss || n <= 0) return AETH_ERR_ARG;
  size_t need = 0;
  aeth_mlp_work_floats(n, &need);
  if (work_floats < need) return AETH_ERR_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  long long off[5];
  layer_offsets(off);
  const int dims[5] = {MLP_IN, MLP_H, MLP_H, MLP_H, MLP_OUT};
  const long long H = MLP_H;
  float* Z[4];
  float* Aact[4];
  float* w = d_work;
  for (int l = 1; l <= 3; ++l) { Z[l] = w; w += (long long)n * H; Aact[l] = w; w += (long long)n * H; }
  float* Yh = w; w += (long long)n * MLP_OUTP;
  float* dY = w; w += (long long)n * MLP_OUTP;
  float* dZa = w; w += (long long)n * H;
  float* dZb = w;
  const int T = 256;
  // forward: Z_l = A_{l-1} W_l^T, + b, act
  const float* prev = d_X;
  long long ldp = MLP_INP;
  for (int l = 0; l < 4; ++l) {
    const int nin = dims[l], nout = dims[l + 1];
    const float* W = d_params + off[l];
    const float* b = W + (long long)nout * nin;
    float* Zo = l < 3 ? Z[l + 1] : Yh;
    float* Ao = l < 3 ? Aact[l + 1] : Yh;
    const long long ldo = l < 3 ? H : MLP_OUTP;
    sgemm(st, n, nout, nin, 1.0f, prev, ldp, 1, W, 1, nin, 0.0f, Zo, ldo);
    k_bias_act<<<(int)(((long long)n * nout + T - 1) / T), T, 0, st>>>(Zo, Ao, b, n, nout, (int)ldo, l < 3);
    prev = Ao;
    ldp = ldo;
  }
  if (cudaMemsetAsync(d_loss, 0, sizeof(float), st) != cudaSuccess) return AETH_ERR_CUDA;
  k_loss<<<(n + T - 1) / T, T, 0, st>>>(Yh, d_Y, dY, n, d_loss);
  // backward
  const float* dZ = dY;
  long long ldz = MLP_OUTP;
  float* bufs[2] = {dZa, dZb};
  for (int l = 3; l >= 0; --l) {
    const int nin = dims[l], nout = dims[l + 1];
    const float* W = d_params + off[l];
    float* gW = d_grad + off[l];
    float* gb = gW + (long long)nout * nin;
    const float* Ain = l > 0 ? Aact[l] : d_X;
    const long long lda = l > 0 ? H : MLP_INP;
    // dW = dZ^T A_in : M = nout, N = nin, K = n
    sgemm(st, nout, nin, n, 1.0f, dZ, 1, ldz, Ain, lda, 1, 0.0f, gW, nin);
    k_colsum<<<nout, 256, 0, st>>>(dZ, gb, n, nout, (int)ldz);
    if (l > 0) {
      float* dA = bufs[l & 1];
      // dA = dZ W : M = n, N = nin, K = nout
      sgemm(st, n, nin, nout, 1.0f, dZ, ldz, 1, W, nin, 1, 0.0f, dA, H);
      const long long tot = (long long)n * H;
      k_dsilu<<<(int)((tot + T - 1) / T), T, 0, st>>>(dA, Z[l], tot);
      dZ = dA;
      ldz = H;
    }
  }
  return cudaGetLastError() == cudaSuccess ? AETH_OK : AETH_ERR_CUDA;
}

extern "C" aeth_status aeth_mlp_adam(float* d_params, const float* d_grad, float* d_m, float* d_v,
                                     long long n, int step, float lr, float beta1, float beta2,
                                     float eps, void* cuda_stream) {
  if (!d_params || !d_grad || !d_m || !d_v || n <= 0 || step < 1) return AETH_ERR_ARG;
  const float c1 = 1.0f - powf(beta1, (float)step), c2 = 1.0f - powf(beta2, (float)step);
  k_adam<<<(int)((n + 255) / 256), 256, 0, (cudaStream_t)cuda_stream>>>(d_params, d_grad, d_m, d_v, n,
                                                                        lr, beta1, beta2, eps, c1, c2);
  return cudaGetLastError() == cudaSuccess ? AETH_OK : AETH_ERR_CUDA;
}

// ------------------------------------------------------------------------
// collect training samples from a context's current state
// ------------------------------------------------------------------------
template <typename R>
static aeth_status collect_T(aeth_ctx* c, int stride, float* X, float* Y, long long cap,
                             long long* n_out) {
  unsigned long long* cnt = (unsigned long long*)(c->arena + c->off_scalars + 448);
  AETH_CK(c, cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), c->stream));
  for (int b = 0; b < (int)c->blocks.size(); ++b) {
    // the stencil reads ghosts: fill them for register A first
    BlockPtrs<R> P = block_ptrs<R>(c, b);
    launch_fill<R>(P, P.reg[0], is_mhd(c) ? NVAR : 5, c->stream);
    const Layout& L = P.L;
    dim3 blk(32, 4, 2), grd((L.n[0] + 31) / 32, (L.n[1] + 3) / 4, (L.n[2] + 1) / 2);
    k_mlp_samples<R><<<grd, blk, 0, c->stream>>>(P, stride, cap, X, Y, cnt, (R)c->cfg.gamma,
                                                 (R)c->cfg.rho_floor, (R)c->cfg.p_floor, is_mhd(c));
  }
  unsigned long long h = 0;
  AETH_CK(c, cudaMemcpyAsync(&h, cnt, sizeof h, cudaMemcpyDeviceToHost, c->stream));
  AETH_CK(c, cudaStreamSynchronize(c->stream));
  if (n_out) *n_out = (long long)std::min<unsigned long long>(h, (unsigned long long)cap);
  return AETH_OK;
}

extern "C" aeth_status aeth_mlp_collect(aeth_ctx* c, int stride, float* d_X, float* d_Y,
                                        long long capacity, long long* n_out) {
  if (!c || !d_X || !d_Y || stride < 1 || capacity < 0) return AETH_ERR_ARG;
  if (!c->finalized) return fail(c, AETH_ERR_STATE, "call aeth_finalize first");
  if (c->cfg.n_dust > 0) return fail(c, AETH_ERR_UNSUPPORTED, "no learned flux for dust runs");
  // the sample stencils take their ghosts from a per-block fill, which
  // knows no linked neighbour (and would rewrite a linked block's face n)
  if (!c->links.empty())
    return fail(c, AETH_ERR_UNSUPPORTED, "training samples come from contexts without linked blocks");
  return c->elem == 8 ? collect_T<double>(c, stride, d_X, d_Y, capacity, n_out)
                      : collect_T<float>(c, stride, d_X, d_Y, capacity, n_out);
}

// ------------------------------------------------------------------------
// BF16 tensor-core inference with per-face checks and HLLD fallback
// ------------------------------------------------------------------------
namespace aeth {

// Device weight block (library-owned): padded BF16 matrices, FP32 biases.
constexpr int LD1 = 24;    // row pitch (bf16) of W1 and of the input tile
constexpr int LDH = 136;   // row pitch (bf16) of W2, W3, W4: conflict-free
constexpr size_t MLP_W1 = 0;
constexpr size_t MLP_W2 = MLP_W1 + 128 * LD1;
constexpr size_t MLP_W3 = MLP_W2 + 128 * LDH;
constexpr size_t MLP_W4 = MLP_W3 + 128 * LDH;
constexpr size_t MLP_NBF16 = MLP_W4 + 8 * LDH;      // bf16 elements
constexpr size_t MLP_NF32 = 3 * 128 + 8;            // biases
constexpr size_t MLP_BYTES = MLP_NBF16 * 2 + MLP_NF32 * 4;
constexpr int MLP_WARPS = 8;
constexpr size_t MLP_SMEM = MLP_BYTES + MLP_WARPS * (32 * LD1 * 2 + 32 * 8 * 4);

__device__ __forceinline__ void mma_bf16(float* d, const unsigned* a, const unsigned* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<unsigned*>(&v);
}

__device__ __forceinline__ unsigned lds32(const __nv_bfloat16* p) {
  return *reinterpret_cast<const unsigned*>(p);
}

// One m-tile (16 faces) through the network.  Fragment layouts of
// m16n8k16 (g = lane / 4, q = lane % 4): A regs (row g | g+8) x (cols 2q |
// 2q+8); B regs (k = 2q | 2q+8, n = g); C (row g | g+8, cols 2q, 2q+1).
// The accumulators of n-tiles 2ks and 2ks+1 are the A fragment of k-step ks
// of the next layer.
__device__ __forceinline__ void mlp_tile(const __nv_bfloat16* __restrict__ sW,
                                         const float* __restrict__ sb,
                                         const __nv_bfloat16* __restrict__ sX, float* __restrict__ sY,
                                         int lane) {
  const int g = lane >> 2, q = lane & 3;
  const __nv_bfloat16* W1 = sW + MLP_W1;
  const __nv_bfloat16* W2 = sW + MLP_W2;
  const __nv_bfloat16* W3 = sW + MLP_W3;
  const __nv_bfloat16* W4 = sW + MLP_W4;
  const float* b1 = sb;
  const float* b2 = sb + 128;
  const float* b3 = sb + 256;
  const float* b4 = sb + 384;
  unsigned A[8][4];
  float C[16][4];
  // layer 1: K = 16 (one k-step)
  A[0][0] = lds32(sX + g * LD1 + 2 * q);
  A[0][1] = lds32(sX + (g + 8) * LD1 + 2 * q);
  A[0][2] = lds32(sX + g * LD1 + 2 * q + 8);
  A[0][3] = lds32(sX + (g + 8) * LD1 + 2 * q + 8);
#pragma unroll
  for (int nt = 0; nt < 16; ++nt) {
    C[nt][0] = C[nt][1] = C[nt][2] = C[nt][3] = 0.0f;
    const unsigned b[2] = {lds32(W1 + (nt * 8 + g) * LD1 + 2 * q),
                           lds32(W1 + (nt * 8 + g) * LD1 + 2 * q + 8)};
    mma_bf16(C[nt], A[0], b);
  }
  auto activate = [&](const float* bias) {
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) {
      const int col = nt * 8 + 2 * q;
      const float v00 = silu_f(C[nt][0] + bias[col]), v01 = silu_f(C[nt][1] + bias[col + 1]);
      const float v10 = silu_f(C[nt][2] + bias[col]), v11 = silu_f(C[nt][3] + bias[col + 1]);
      const int ks = nt >> 1;
      if ((nt & 1) == 0) { A[ks][0] = pack_bf16(v00, v01); A[ks][1] = pack_bf16(v10, v11); }
      else { A[ks][2] = pack_bf16(v00, v01); A[ks][3] = pack_bf16(v10, v11); }
    }
  };
  activate(b1);
  // layers 2 and 3: K = 128
  const __nv_bfloat16* Wh[2] = {W2, W3};
  const float* bh[2] = {b2, b3};
#pragma unroll
  for (int l = 0; l < 2; ++l) {
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) {
      C[nt][0] = C[nt][1] = C[nt][2] = C[nt][3] = 0.0f;
      const __nv_bfloat16* row = Wh[l] + (nt * 8 + g) * LDH + 2 * q;
#pragma unroll
      for (int ks = 0; ks < 8; ++ks) {
        const unsigned b[2] = {lds32(row + ks * 16), lds32(row + ks * 16 + 8)};
        mma_bf16(C[nt], A[ks], b);
      }
    }
    activate(bh[l]);
  }
  // layer 4: one n-tile of 8 outputs (7 used), linear
  float D[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  const __nv_bfloat16* row4 = W4 + g * LDH + 2 * q;
#pragma unroll
  for (int ks = 0; ks < 8; ++ks) {
    const unsigned b[2] = {lds32(row4 + ks * 16), lds32(row4 + ks * 16 + 8)};
    mma_bf16(D, A[ks], b);
  }
  sY[g * 8 + 2 * q] = D[0] + b4[2 * q];
  sY[g * 8 + 2 * q + 1] = D[1] + b4[2 * q + 1];
  sY[(g + 8) * 8 + 2 * q] = D[2] + b4[2 * q];
  sY[(g + 8) * 8 + 2 * q + 1] = D[3] + b4[2 * q + 1];
}

// Faces of direction D of one block: states from the dump arrays, fluxes
// into the same output arrays as the HLLD flux pass.
template <typename R, int D>
__global__ void __launch_bounds__(MLP_WARPS * 32, 1)
    k_mlp_flux(BlockPtrs<R> P, const R* __restrict__ fs, const void* __restrict__ wdev, R gamma,
               R tau, int mhd, unsigned long long* fallbacks) {
  extern __shared__ __align__(16) unsigned char smem[];
  __nv_bfloat16* sW = reinterpret_cast<__nv_bfloat16*>(smem);
  float* sb = reinterpret_cast<float*>(smem + MLP_NBF16 * 2);
  unsigned char* wbase = smem + MLP_BYTES;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __nv_bfloat16* sX = reinterpret_cast<__nv_bfloat16*>(wbase + warp * (32 * LD1 * 2 + 32 * 8 * 4));
  float* sY = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(sX) + 32 * LD1 * 2);
  // stage the weights (16-byte copies)
  {
    const uint4* src = reinterpret_cast<const uint4*>(wdev);
    uint4* dst = reinterpret_cast<uint4*>(smem);
    for (size_t t = threadIdx.x; t < MLP_BYTES / 16; t += blockDim.x) dst[t] = src[t];
  }
  __syncthreads();
  const Layout L = P.L;
  const long long pitch = P.pitch;
  const int nseg = (L.n[0] + 2 + 31) / 32;
  const long long nwork = (long long)nseg * (L.n[1] + 2) * (L.n[2] + 2);
  constexpr int T1 = (D + 1) % 3, T2 = (D + 2) % 3;
  unsigned long long fb = 0;
  for (long long wk = (long long)blockIdx.x * MLP_WARPS + warp; wk < nwork;
       wk += (long long)gridDim.x * MLP_WARPS) {
    const int seg = (int)(wk % nseg);
    const long long row = wk / nseg;
    const int j = (int)(row % (L.n[1] + 2)) - 1, k = (int)(row / (L.n[1] + 2)) - 1;
    const int i = seg * 32 + lane - 1;
    int c3[3] = {i, j, k};
    bool valid = i <= L.n[0] && c3[D] >= 0;
    const long long fc = L.idx(min(i, L.n[0]), j, k);
    R wl[7], wr[7], bn = R(0);
    if (valid) {
#pragma unroll
      for (int q = 0; q < 7; ++q) {
        wl[q] = fs[(D * 15 + q) * pitch + fc];
        wr[q] = fs[(D * 15 + 7 + q) * pitch + fc];
      }
      bn = fs[(D * 15 + 14) * pitch + fc];
    } else {
#pragma unroll
      for (int q = 0; q < 7; ++q) wl[q] = wr[q] = R(0);
      wl[0] = wr[0] = R(1); wl[4] = wr[4] = R(1);
    }
    float x[16];
    const FaceScale sc = mlp_features(wl, wr, bn, gamma, x);
#pragma unroll
    for (int q = 0; q < 16; q += 2)
      *reinterpret_cast<unsigned*>(sX + lane * LD1 + q) = pack_bf16(x[q], x[q + 1]);
    __syncwarp();
    mlp_tile(sW, sb, sX, sY, lane);
    mlp_tile(sW, sb, sX + 16 * LD1, sY + 16 * 8, lane);
    __syncwarp();
    float k7[7];
    mlp_scale_out(sc, (float)gamma, k7);
    float y[7];
#pragma unroll
    for (int q = 0; q < 7; ++q) y[q] = sY[lane * 8 + q];
    __syncwarp();
    if (!valid) continue;
    R F[7];
    if (!mlp_compose(gamma, wl, wr, bn, y, k7, tau, mhd != 0, F)) {
      hlld(gamma, wl, wr, bn, F);
      ++fb;
    }
    R* sbp = P.w[0];
    R* f = sbp + (8 + 5 * D) * pitch + fc;
    f[0] = F[0];
    f[(1 + D) * pitch] = F[1];
    f[(1 + T1) * pitch] = F[2];
    f[(1 + T2) * pitch] = F[3];
    f[4 * pitch] = F[4];
    R* e = sbp + (23 + 2 * D) * pitch + fc;
    e[0] = F[6];
    e[pitch] = -F[5];
  }
  for (int o = 16; o > 0; o >>= 1) fb += __shfl_xor_sync(0xffffffffu, fb, o);
  if (lane == 0 && fb) atomicAdd(fallbacks, fb);
}

// Tensor-core forward of feature rows X[n][16] -> Y[n][8] (dimensionless).
__global__ void __launch_bounds__(MLP_WARPS * 32, 1)
    k_mlp_infer(const float* __restrict__ X, float* __restrict__ Y, int n,
                const void* __restrict__ wdev) {
  extern __shared__ __align__(16) unsigned char smem[];
  __nv_bfloat16* sW = reinterpret_cast<__nv_bfloat16*>(smem);
  float* sb = reinterpret_cast<float*>(smem + MLP_NBF16 * 2);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* wbase = smem + MLP_BYTES;
  __nv_bfloat16* sX = reinterpret_cast<__nv_bfloat16*>(wbase + warp * (32 * LD1 * 2 + 32 * 8 * 4));
  float* sY = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(sX) + 32 * LD1 * 2);
  {
    const uint4* src = reinterpret_cast<const uint4*>(wdev);
    uint4* dst = reinterpret_cast<uint4*>(smem);
    for (size_t t = threadIdx.x; t < MLP_BYTES / 16; t += blockDim.x) dst[t] = src[t];
  }
  __syncthreads();
  for (int base = (blockIdx.x * MLP_WARPS + warp) * 32; base < n; base += gridDim.x * MLP_WARPS * 32) {
    const int r = base + lane;
#pragma unroll
    for (int q = 0; q < 16; q += 2) {
      const float a = r < n ? X[(long long)r * 16 + q] : 0.0f;
      const float b = r < n ? X[(long long)r * 16 + q + 1] : 0.0f;
      *reinterpret_cast<unsigned*>(sX + lane * LD1 + q) = pack_bf16(a, b);
    }
    __syncwarp();
    mlp_tile(sW, sb, sX, sY, lane);
    mlp_tile(sW, sb, sX + 16 * LD1, sY + 16 * 8, lane);
    __syncwarp();
    if (r < n)
      for (int q = 0; q < 8; ++q) Y[(long long)r * 8 + q] = sY[lane * 8 + q];
    __syncwarp();
  }
}

template <typename R>
void mlp_flux_pass_tc(aeth_ctx* c, int block);

template <typename R>
void mlp_flux_pass(aeth_ctx* c, int block) {
  if (c->cfg.mlp_engine == AETH_MLP_TCGEN05) {
    mlp_flux_pass_tc<R>(c, block);
    return;
  }
  const BlockPtrs<R> P = block_ptrs<R>(c, block);
  const Layout& L = P.L;
  const long long nseg = (L.n[0] + 2 + 31) / 32;
  const long long nwork = nseg * (L.n[1] + 2) * (L.n[2] + 2);
  const int grid = (int)std::max(1LL, std::min(nwork / MLP_WARPS + 1, 2LL * c->num_sms));
  const R* fs = P.fstate;
  const R g = (R)c->cfg.gamma;
  const R tau = (R)(c->cfg.mlp_tau > 0 ? c->cfg.mlp_tau : 0.25);
  const int mhd = is_mhd(c);
  k_mlp_flux<R, 0><<<grid, MLP_WARPS * 32, MLP_SMEM, c->stream>>>(P, fs, c->d_mlp, g, tau, mhd, c->d_fallback);
  k_mlp_flux<R, 1><<<grid, MLP_WARPS * 32, MLP_SMEM, c->stream>>>(P, fs, c->d_mlp, g, tau, mhd, c->d_fallback);
  k_mlp_flux<R, 2><<<grid, MLP_WARPS * 32, MLP_SMEM, c->stream>>>(P, fs, c->d_mlp, g, tau, mhd, c->d_fallback);
  c->n_launch += 3;
}
template void mlp_flux_pass<float>(aeth_ctx*, int);
template void mlp_flux_pass<double>(aeth_ctx*, int);

aeth_status mlp_prepare(aeth_ctx* c) {
  for (int D = 0; D < 3; ++D) {
    cudaError_t e = D == 0 ? cudaFuncSetAttribute(k_mlp_flux<float, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MLP_SMEM)
                  : D == 1 ? cudaFuncSetAttribute(k_mlp_flux<float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MLP_SMEM)
                           : cudaFuncSetAttribute(k_mlp_flux<float, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MLP_SMEM);
    if (e != cudaSuccess) return fail(c, AETH_ERR_CUDA, "smem attribute: %s", cudaGetErrorString(e));
    e = D == 0 ? cudaFuncSetAttribute(k_mlp_flux<double, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MLP_SMEM)
      : D == 1 ? cudaFuncSetAttribute(k_mlp_flux<double, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MLP_SMEM)
               : cudaFuncSetAttribute(k_mlp_flux<double, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MLP_SMEM);
    if (e != cudaSuccess) return fail(c, AETH_ERR_CUDA, "smem attribute: %s", cudaGetErrorString(e));
  }
  cudaError_t e = cudaFuncSetAttribute(k_mlp_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MLP_SMEM);
  if (e != cudaSuccess) return fail(c, AETH_ERR_CUDA, "smem attribute: %s", cudaGetErrorString(e));
  return AETH_OK;
}

}  // namespace aeth

namespace aeth {
std::vector<unsigned char> tc_weight_image(const float* params);
aeth_status mlp_tc_prepare(aeth_ctx* c);
}  // namespace aeth

extern "C" aeth_status aeth_load_mlp(aeth_ctx* c, const float* params, size_t n) {
  if (!c || !params) return AETH_ERR_ARG;
  if (n != (size_t)MLP_NPARAM)
    return fail(c, AETH_ERR_ARG, "expected %lld parameters, got %zu", MLP_NPARAM, n);
  long long off[5];
  layer_offsets(off);
  std::vector<__nv_bfloat16> wb(MLP_NBF16, __float2bfloat16(0.0f));
  std::vector<float> bias(MLP_NF32, 0.0f);
  auto put = [&](size_t base, int ld, int layer, int nout, int nin) {
    const float* W = params + off[layer];
    for (int o = 0; o < nout; ++o)
      for (int i = 0; i < nin; ++i) wb[base + (size_t)o * ld + i] = __float2bfloat16(W[(size_t)o * nin + i]);
  };
  put(MLP_W1, LD1, 0, MLP_H, MLP_IN);
  put(MLP_W2, LDH, 1, MLP_H, MLP_H);
  put(MLP_W3, LDH, 2, MLP_H, MLP_H);
  put(MLP_W4, LDH, 3, MLP_OUT, MLP_H);
  const int dims[5] = {MLP_IN, MLP_H, MLP_H, MLP_H, MLP_OUT};
  for (int l = 0; l < 4; ++l) {
    const float* b = params + off[l] + (long long)dims[l + 1] * dims[l];
    for (int o = 0; o < dims[l + 1]; ++o) bias[l * 128 + o] = b[o];
  }
  if (!c->d_mlp) {
    if (cudaMalloc(&c->d_mlp, MLP_BYTES) != cudaSuccess)
      return fail(c, AETH_ERR_OOM, "cannot allocate the network weights");
  }
  AETH_CK(c, cudaMemcpyAsync(c->d_mlp, wb.data(), MLP_NBF16 * 2, cudaMemcpyHostToDevice, c->stream));
  AETH_CK(c, cudaMemcpyAsync((char*)c->d_mlp + MLP_NBF16 * 2, bias.data(), MLP_NF32 * 4,
                             cudaMemcpyHostToDevice, c->stream));
  AETH_CK(c, cudaStreamSynchronize(c->stream));
  {
    // the tcgen05 path's weight image (core-matrix layout)
    std::vector<unsigned char> img = tc_weight_image(params);
    if (!c->d_mlp_tc && cudaMalloc(&c->d_mlp_tc, img.size()) != cudaSuccess)
      return fail(c, AETH_ERR_OOM, "cannot allocate the network weights");
    AETH_CK(c, cudaMemcpyAsync(c->d_mlp_tc, img.data(), img.size(), cudaMemcpyHostToDevice, c->stream));
    AETH_CK(c, cudaStreamSynchronize(c->stream));
    aeth_status s = mlp_tc_prepare(c);
    if (s != AETH_OK) return s;
  }
  c->mlp_n = n;
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  return mlp_prepare(c);
}

extern "C" aeth_status aeth_mlp_infer(aeth_ctx* c, const float* d_X, float* d_Y, int n) {
  if (!c || !d_X || !d_Y || n < 0) return AETH_ERR_ARG;
  if (!c->d_mlp) return fail(c, AETH_ERR_STATE, "call aeth_load_mlp first");
  if (n == 0) return AETH_OK;
  const int grid = std::max(1, std::min((n + MLP_WARPS * 32 - 1) / (MLP_WARPS * 32), 2 * c->num_sms));
  k_mlp_infer<<<grid, MLP_WARPS * 32, MLP_SMEM, c->stream>>>(d_X, d_Y, n, c->d_mlp);
  AETH_CK(c, cudaGetLastError());
  c->n_launch += 1;
  return AETH_OK;
}
