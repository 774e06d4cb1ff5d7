// Learned-flux network on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// A CTA holds one copy of the BF16 weights in shared memory and NWG
// independent warpgroups; each warpgroup pushes tiles of 128 rows (faces)
// through the 14(16) -> 128 -> 128 -> 128 -> 7(16) network:
//   * operands in shared memory, no swizzle, K-major "core matrices" of
//     8 rows x 8 BF16 (128 contiguous bytes); core matrices adjacent in K are
//     128 B apart (leading byte offset), 8-row groups K/8 * 128 B apart
//     (stride byte offset);
//   * one thread of the warpgroup issues tcgen05.mma (M = 128, N = 128 or 16,
//     K = 16 per instruction, BF16 x BF16 -> FP32) into the warpgroup's 128
//     TMEM columns and commits to the warpgroup's mbarrier;
//   * each warp reads its 32 TMEM lanes (= its 32 rows) back with tcgen05.ld,
//     adds the bias, applies SiLU and stores the next layer's A tile (BF16)
//     to shared memory with 16-byte, bank-conflict-free stores.
// While one warpgroup waits for its MMAs the others run their epilogues, the
// face features and the acceptance test, so the tensor pipe and the
// FP32/MUFU pipes overlap.
// Every mbarrier wait is bounded (probes and wall time): on time-out the
// warpgroup stops, raises the time-out status bit, drains its MMAs (again
// bounded) and the CTA still releases its TMEM.
#include <cuda_bf16.h>

#include <cstring>
#include <vector>

#include "mlp_face.cuh"
#include "runtime.hpp"

namespace aeth {
namespace tc {

constexpr int TM = 128;   // rows per warpgroup tile (TMEM lanes)
// shared-memory image of the network (bytes)
constexpr int OFF_W1 = 0;                        // B tile [128 n][16 k]
constexpr int OFF_W2 = OFF_W1 + 128 * 16 * 2;    // B tile [128 n][128 k]
constexpr int OFF_W3 = OFF_W2 + 128 * 128 * 2;
constexpr int OFF_W4 = OFF_W3 + 128 * 128 * 2;   // B tile [16 n][128 k]
constexpr int OFF_BIAS = OFF_W4 + 16 * 128 * 2;  // 3 x 128 + 16 floats
constexpr int WBYTES = OFF_BIAS + 2048;
// per warpgroup: A tile [128 m][128 k] and input tile [128 m][16 k]
constexpr int WG_A = 0;
constexpr int WG_X = 128 * 128 * 2;
constexpr int WG_BYTES = WG_X + 128 * 16 * 2;

__host__ __device__ constexpr int smem_bytes(int nwg) { return WBYTES + nwg * WG_BYTES + 128; }

// byte offset of element (row r, col k) in a K-major tile with K columns
__host__ __device__ __forceinline__ int core_off(int r, int k, int K) {
  return ((r >> 3) * (K >> 3) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor (no swizzle)
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version of this architecture
  return d;
}

// instruction descriptor: kind::f16, A = B = BF16, D = FP32, K-major A, B
__host__ __device__ constexpr uint32_t idesc(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t id,
                                    uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}

__device__ __forceinline__ void commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// bounded wait for the phase of parity `parity`: at most ~2^20 probes and
// ~0.5 s of wall time
__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity) {
  const unsigned long long t0 = now_ns();
  for (int it = 0; it < (1 << 20); ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 255) == 255 && now_ns() - t0 > 500000000ull) return false;
  }
  return false;
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// barrier over the 128 threads of one warpgroup, AND-reducing v
__device__ __forceinline__ bool wg_sync_and(int id, bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred pi, po;\n\tsetp.ne.u32 pi, %1, 0;\n\t"
      "bar.red.and.pred po, %2, 128, pi;\n\tselp.u32 %0, 1, 0, po;\n\t}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(id)
      : "memory");
  return r != 0;
}

// 32 (resp. 8) FP32 columns of this warp's 32 TMEM lanes
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
        "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
        "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int q = 0; q < 32; ++q) v[q] = __uint_as_float(r[q]);
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                 "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = __uint_as_float(r[q]);
}

// SiLU z * sigma(z) with sigma(z) = (1 + tanh(z / 2)) / 2: one MUFU op
__device__ __forceinline__ float silu_t(float z) {
  float t;
  asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(0.5f * z));
  return z * fmaf(0.5f, t, 0.5f);
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&h);
}

// One warpgroup's state.
struct WG {
  unsigned char* sA;   // A tile (layers 2..4)
  unsigned char* sX;   // input tile (layer 1)
  uint32_t tmem;       // first of the warpgroup's 128 columns, lane 0
  uint32_t lanes;      // this warp's lane quarter in the TMEM address
  uint32_t bar;        // the warpgroup's mbarrier
  uint32_t phase;
  int wid;             // thread index in the warpgroup = tile row
  int bar_id;          // named barrier of the warpgroup
};

// The network on the warpgroup's 128 rows: x = this thread's 16 inputs,
// y = its 8 outputs.  Returns false, uniformly over the warpgroup, if an
// MMA wait timed out (y is then undefined).
__device__ __forceinline__ bool forward(const unsigned char* sm, WG& g, const float* x, float* y) {
  {
    uint4 lo = make_uint4(pack2(x[0], x[1]), pack2(x[2], x[3]), pack2(x[4], x[5]), pack2(x[6], x[7]));
    uint4 hi = make_uint4(pack2(x[8], x[9]), pack2(x[10], x[11]), pack2(x[12], x[13]), pack2(x[14], x[15]));
    *reinterpret_cast<uint4*>(g.sX + core_off(g.wid, 0, 16)) = lo;
    *reinterpret_cast<uint4*>(g.sX + core_off(g.wid, 8, 16)) = hi;
  }
  const float* bias = reinterpret_cast<const float*>(sm + OFF_BIAS);
  const uint32_t sA = smem_u32(g.sA), sX = smem_u32(g.sX);
  bool ok = true;
#pragma unroll 1
  for (int layer = 0; layer < 4; ++layer) {
    // the tile written by every thread (generic proxy) and every warp's
    // TMEM reads complete before the next MMA
    fence_async_smem();
    fence_before();
    ok = wg_sync_and(g.bar_id, ok);
    fence_after();
    if (!ok) return false;
    if (g.wid == 0) {
      if (layer == 0) {
        mma(g.tmem, sdesc(sX, 128, 256), sdesc(smem_u32(sm + OFF_W1), 128, 256), idesc(128, 128), 0);
      } else {
        const uint32_t sB = smem_u32(sm + (layer == 1 ? OFF_W2 : (layer == 2 ? OFF_W3 : OFF_W4)));
        const uint32_t id = layer == 3 ? idesc(128, 16) : idesc(128, 128);
#pragma unroll
        for (int ks = 0; ks < 8; ++ks)
          mma(g.tmem, sdesc(sA + ks * 256, 128, 2048), sdesc(sB + ks * 256, 128, 2048), id, ks > 0);
      }
      commit(g.bar);
    }
    ok = wait_bar(g.bar, g.phase);
    g.phase ^= 1u;
    fence_after();
    if (!ok) continue;   // the next barrier makes the failure uniform
    if (layer < 3) {
      const float* b = bias + layer * 128;
#pragma unroll 1
      for (int cb = 0; cb < 4; ++cb) {
        float v[32];
        tmem_ld32(g.tmem + g.lanes + cb * 32, v);
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          const float* bb = b + cb * 32 + h * 8;
          const float* vv = v + h * 8;
          uint4 pk = make_uint4(pack2(silu_t(vv[0] + bb[0]), silu_t(vv[1] + bb[1])),
                                pack2(silu_t(vv[2] + bb[2]), silu_t(vv[3] + bb[3])),
                                pack2(silu_t(vv[4] + bb[4]), silu_t(vv[5] + bb[5])),
                                pack2(silu_t(vv[6] + bb[6]), silu_t(vv[7] + bb[7])));
          *reinterpret_cast<uint4*>(g.sA + core_off(g.wid, cb * 32 + h * 8, 128)) = pk;
        }
      }
    } else {
      tmem_ld8(g.tmem + g.lanes, y);
#pragma unroll
      for (int q = 0; q < 8; ++q) y[q] += bias[384 + q];
    }
  }
  fence_before();
  ok = wg_sync_and(g.bar_id, ok);
  fence_after();
  return ok;
}

// CTA prologue: weights to shared memory, one mbarrier per warpgroup, TMEM
// columns for all warpgroups.  Returns this thread's warpgroup state.
template <int NWG>
__device__ __forceinline__ WG setup(unsigned char* sm, const unsigned char* __restrict__ wimg) {
  constexpr int COLS = NWG * 128;
  static_assert(COLS == 128 || COLS == 256 || COLS == 512, "TMEM allocation is a power of 2");
  const int tid = threadIdx.x, warp = tid >> 5, wg = tid >> 7;
  {
    const uint4* s = reinterpret_cast<const uint4*>(wimg);
    uint4* d = reinterpret_cast<uint4*>(sm);
    for (int t = tid; t < WBYTES / 16; t += blockDim.x) d[t] = s[t];
  }
  unsigned char* misc = sm + WBYTES + NWG * WG_BYTES;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(misc + 64);
  if (tid < NWG) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(misc + 8 * tid)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                 "r"(COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  WG g;
  g.sA = sm + WBYTES + wg * WG_BYTES + WG_A;
  g.sX = sm + WBYTES + wg * WG_BYTES + WG_X;
  g.tmem = *tslot + (uint32_t)(wg * 128);
  g.lanes = (uint32_t)((warp & 3) * 32) << 16;
  g.bar = smem_u32(misc + 8 * wg);
  g.phase = 0;
  g.wid = tid & 127;
  g.bar_id = 1 + wg;
  return g;
}

// CTA epilogue: a warpgroup that timed out raises the status bit and drains
// its MMAs (bounded); then the TMEM columns are released.
template <int NWG>
__device__ __forceinline__ void teardown(unsigned char* sm, WG& g, bool ok, int* status) {
  if (!ok && g.wid == 0) {
    atomicOr(status, ST_TIMEOUT);
    wait_bar(g.bar, g.phase ^ 1u);
  }
  unsigned char* misc = sm + WBYTES + NWG * WG_BYTES;
  const uint32_t base = *reinterpret_cast<uint32_t*>(misc + 64);
  fence_before();
  __syncthreads();
  fence_after();
  if ((threadIdx.x >> 5) == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(base), "r"(NWG * 128)
                 : "memory");
}

constexpr int NWG_F32 = 4;   // 512 threads, <= 128 registers, 512 TMEM columns
constexpr int NWG_F64 = 2;   // FP64 face states need more registers

}  // namespace tc

// X[n][16] -> Y[n][8] (dimensionless rows).
__global__ void __launch_bounds__(tc::NWG_F32 * 128, 1)
    k_mlp_tc(const float* __restrict__ X, float* __restrict__ Y, int n,
             const unsigned char* __restrict__ wimg, int* status) {
  using namespace tc;
  constexpr int NWG = NWG_F32;
  extern __shared__ __align__(1024) unsigned char sm[];
  WG g = setup<NWG>(sm, wimg);
  const int wg = threadIdx.x >> 7;
  bool ok = true;
  for (int tile = blockIdx.x * NWG + wg; tile * TM < n; tile += gridDim.x * NWG) {
    const int r = tile * TM + g.wid;
    float x[16];
    if (r < n) {
      const float4* src = reinterpret_cast<const float4*>(X + (long long)r * 16);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 t = src[q];
        x[4 * q] = t.x; x[4 * q + 1] = t.y; x[4 * q + 2] = t.z; x[4 * q + 3] = t.w;
      }
    } else {
#pragma unroll
      for (int q = 0; q < 16; ++q) x[q] = 0.0f;
    }
    float y[8];
    ok = forward(sm, g, x, y);
    if (!ok) break;
    if (r < n) {
      float4* dst = reinterpret_cast<float4*>(Y + (long long)r * 8);
      dst[0] = make_float4(y[0], y[1], y[2], y[3]);
      dst[1] = make_float4(y[4], y[5], y[6], y[7]);
    }
  }
  teardown<NWG>(sm, g, ok, status);
}

// Learned flux of the faces of direction D of one block (the tcgen05 twin
// of the mma.sync flux kernel): face states from the dump arrays, network,
// acceptance test, HLLD on rejected faces, fluxes and face EMFs into the
// arrays of the HLLD flux pass.  A warpgroup tile is 4 work units of 32
// faces along x.
template <typename R, int D, int NWG>
__global__ void __launch_bounds__(NWG * 128, 1)
    k_mlp_flux_tc(BlockPtrs<R> P, const R* __restrict__ fs, const unsigned char* __restrict__ wimg,
                  R gamma, R tau, int mhd, unsigned long long* fallbacks, int* status) {
  using namespace tc;
  extern __shared__ __align__(1024) unsigned char sm[];
  WG g = setup<NWG>(sm, wimg);
  const int wg = threadIdx.x >> 7, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const Layout L = P.L;
  const long long pitch = P.pitch;
  const int nseg = (L.n[0] + 2 + 31) / 32;
  const long long nwork = (long long)nseg * (L.n[1] + 2) * (L.n[2] + 2);
  const long long ntile = (nwork + 3) / 4;
  constexpr int T1 = (D + 1) % 3, T2 = (D + 2) % 3;
  unsigned long long fb = 0;
  bool ok = true;
  for (long long t = (long long)blockIdx.x * NWG + wg; t < ntile; t += (long long)gridDim.x * NWG) {
    const long long wk = t * 4 + (warp & 3);
    bool valid = wk < nwork;
    const long long wkc = valid ? wk : 0;
    const int seg = (int)(wkc % nseg);
    const long long row = wkc / nseg;
    const int j = (int)(row % (L.n[1] + 2)) - 1, k = (int)(row / (L.n[1] + 2)) - 1;
    const int i = seg * 32 + lane - 1;
    const int c3[3] = {i, j, k};
    valid = valid && i <= L.n[0] && c3[D] >= 0;
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
    float y[8];
    ok = forward(sm, g, x, y);
    if (!ok) break;   // uniform over the warpgroup
    if (!valid) continue;
    float k7[7];
    mlp_scale_out(sc, (float)gamma, k7);
    R F[7];
#pragma unroll
    for (int q = 0; q < 7; ++q) F[q] = (R)(y[q] * k7[q]);
    if (!mhd) F[5] = F[6] = R(0);
    if (!mlp_accept(gamma, wl, wr, bn, F, k7, tau)) {
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
  teardown<NWG>(sm, g, ok, status);
}

template <typename R>
static constexpr int nwg_of() {
  return sizeof(R) == 4 ? tc::NWG_F32 : tc::NWG_F64;
}

template <typename R>
void mlp_flux_pass_tc(aeth_ctx* c, int block) {
  constexpr int NWG = nwg_of<R>();
  const BlockPtrs<R> P = block_ptrs<R>(c, block);
  const Layout& L = P.L;
  const long long nseg = (L.n[0] + 2 + 31) / 32;
  const long long ntile = (nseg * (L.n[1] + 2) * (L.n[2] + 2) + 3) / 4;
  // one CTA per SM (shared memory and TMEM columns)
  const int grid = (int)std::max(1LL, std::min((ntile + NWG - 1) / NWG, (long long)c->num_sms));
  const R g = (R)c->cfg.gamma;
  const R tau = (R)(c->cfg.mlp_tau > 0 ? c->cfg.mlp_tau : 0.25);
  const int mhd = is_mhd(c);
  const unsigned char* w = (const unsigned char*)c->d_mlp_tc;
  constexpr int SM = tc::smem_bytes(NWG);
  k_mlp_flux_tc<R, 0, NWG><<<grid, NWG * 128, SM, c->stream>>>(P, P.fstate, w, g, tau, mhd, c->d_fallback, c->d_status);
  k_mlp_flux_tc<R, 1, NWG><<<grid, NWG * 128, SM, c->stream>>>(P, P.fstate, w, g, tau, mhd, c->d_fallback, c->d_status);
  k_mlp_flux_tc<R, 2, NWG><<<grid, NWG * 128, SM, c->stream>>>(P, P.fstate, w, g, tau, mhd, c->d_fallback, c->d_status);
  c->n_launch += 3;
}
template void mlp_flux_pass_tc<float>(aeth_ctx*, int);
template void mlp_flux_pass_tc<double>(aeth_ctx*, int);

// Host: the network's parameters (W_l[out][in], b_l per layer) as the
// shared-memory image above.
std::vector<unsigned char> tc_weight_image(const float* params) {
  using namespace tc;
  std::vector<unsigned char> img(WBYTES, 0);
  auto put = [&](int off, int ld_k, const float* W, int nout, int nin) {
    for (int o = 0; o < nout; ++o)
      for (int i = 0; i < nin; ++i) {
        __nv_bfloat16 h = __float2bfloat16(W[(size_t)o * nin + i]);
        memcpy(&img[off + core_off(o, i, ld_k)], &h, 2);
      }
  };
  const int dims[5] = {14, 128, 128, 128, 7};
  size_t off = 0;
  const int woff[4] = {OFF_W1, OFF_W2, OFF_W3, OFF_W4};
  const int ldk[4] = {16, 128, 128, 128};
  float* bias = reinterpret_cast<float*>(img.data() + OFF_BIAS);
  for (int l = 0; l < 4; ++l) {
    const int nin = dims[l], nout = dims[l + 1];
    put(woff[l], ldk[l], params + off, nout, nin);
    off += (size_t)nout * nin;
    for (int o = 0; o < nout; ++o) bias[l * 128 + o] = params[off + o];
    off += nout;
  }
  return img;
}

template <typename K>
static cudaError_t big_smem(K kern, int bytes) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
}

aeth_status mlp_tc_prepare(aeth_ctx* c) {
  using namespace tc;
  const int s32 = smem_bytes(NWG_F32), s64 = smem_bytes(NWG_F64);
  cudaError_t e = big_smem(k_mlp_tc, s32);
  if (e == cudaSuccess) e = big_smem(k_mlp_flux_tc<float, 0, NWG_F32>, s32);
  if (e == cudaSuccess) e = big_smem(k_mlp_flux_tc<float, 1, NWG_F32>, s32);
  if (e == cudaSuccess) e = big_smem(k_mlp_flux_tc<float, 2, NWG_F32>, s32);
  if (e == cudaSuccess) e = big_smem(k_mlp_flux_tc<double, 0, NWG_F64>, s64);
  if (e == cudaSuccess) e = big_smem(k_mlp_flux_tc<double, 1, NWG_F64>, s64);
  if (e == cudaSuccess) e = big_smem(k_mlp_flux_tc<double, 2, NWG_F64>, s64);
  if (e != cudaSuccess) return fail(c, AETH_ERR_CUDA, "tcgen05 network smem attribute: %s", cudaGetErrorString(e));
  return AETH_OK;
}

}  // namespace aeth

extern "C" aeth_status aeth_mlp_infer_tc(aeth_ctx* c, const float* d_X, float* d_Y, int n) {
  using namespace aeth;
  if (!c || !d_X || !d_Y || n < 0) return AETH_ERR_ARG;
  if (!c->d_mlp_tc) return fail(c, AETH_ERR_STATE, "call aeth_load_mlp first");
  if (((uintptr_t)d_X | (uintptr_t)d_Y) & 15)
    return fail(c, AETH_ERR_ARG, "X and Y must be 16-byte aligned");
  if (n == 0) return AETH_OK;
  const int tiles = (n + tc::TM - 1) / tc::TM;
  const int grid = std::max(1, std::min((tiles + tc::NWG_F32 - 1) / tc::NWG_F32, c->num_sms));
  k_mlp_tc<<<grid, tc::NWG_F32 * 128, tc::smem_bytes(tc::NWG_F32), c->stream>>>(
      d_X, d_Y, n, (const unsigned char*)c->d_mlp_tc, c->d_status);
  AETH_CK(c, cudaGetLastError());
  c->n_launch += 1;
  return AETH_OK;
}
