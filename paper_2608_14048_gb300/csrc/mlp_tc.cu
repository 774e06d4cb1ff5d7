// Learned-flux network on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// A CTA holds one copy of the BF16 weights in shared memory and, by default
// (AETH_TC_TPW = 1), four independent warpgroups of 128 threads; each
// warpgroup pushes one 128-row tile (128 faces) at a time through the
// 14(16) -> 128 -> 128 -> 128 -> 7(16) network, so four tiles are in flight
// per CTA (512 TMEM columns):
//   * operands in shared memory, no swizzle, K-major "core matrices" of
//     8 rows x 8 BF16 (128 contiguous bytes); core matrices adjacent in K are
//     128 B apart (leading byte offset), 8-row groups K/8 * 128 B apart
//     (stride byte offset);
//   * one thread of the warpgroup issues tcgen05.mma (M = 128, N = 128 or 16,
//     K = 16 per instruction, BF16 x BF16 -> FP32) into the tile's 128 TMEM
//     columns and commits to the tile's mbarrier;
//   * the hidden layers' weights and biases are stored halved (exact in
//     BF16), so the accumulator is h = z / 2 of the pre-activation z; the
//     biases enter the accumulator through the MMA: the input tile carries
//     ones in its padding columns 14 and 15, W1 carries the bias there as a
//     BF16 hi + lo pair, and layers 2 and 3 take one more K = 16 step with
//     the input tile as A and a [128][16] bias tile (hi, lo in columns 14,
//     15) as B;
//   * each warp reads its 32 TMEM lanes (= its 32 rows) back with tcgen05.ld
//     (the next 32 columns in flight while the current ones are used),
//     applies SiLU and stores the next layer's A tile (BF16) to shared
//     memory with 16-byte, bank-conflict-free stores.
// The tensor pipe and the MUFU/FP32 pipes overlap across the four
// warpgroups: while one warpgroup runs its SiLU epilogue, the tensor core
// runs another's next layer.  The alternative build AETH_TC_TPW = 2 gives
// two warpgroups of two ping-pong tiles each (one tile's MMAs overlap the
// same warpgroup's SiLU on the other); it measured slower than four
// single-tile warpgroups and is kept selectable only.
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
constexpr int OFF_BB2 = OFF_W4 + 16 * 128 * 2;   // bias tiles [128 n][16 k]
constexpr int OFF_BB3 = OFF_BB2 + 128 * 16 * 2;
constexpr int OFF_B4 = OFF_BB3 + 128 * 16 * 2;   // output bias, 16 floats
constexpr int WBYTES = OFF_B4 + 64;
// per warpgroup: A tile [128 m][128 k] and input tile [128 m][16 k]
constexpr int WG_A = 0;
constexpr int WG_X = 128 * 128 * 2;
constexpr int WG_BYTES = WG_X + 128 * 16 * 2;

__host__ __device__ constexpr int smem_bytes(int tiles) { return WBYTES + tiles * WG_BYTES + 128; }

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

// 32 FP32 columns of this warp's 32 TMEM lanes.  The load is asynchronous:
// tmem_wait32 completes it and names the registers as in/out operands, so
// no use of them can be scheduled before the wait.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait32(uint32_t (&r)[32]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;\n"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
               :
               : "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                 "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                 "+r"(r[6]), "+r"(r[7])
               :
               : "memory");
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = __uint_as_float(r[q]);
}

// SiLU of the pre-activation z from the accumulator h = z / 2:
//   silu(z) = z sigma(z) = h (1 + tanh h) = h + h tanh h,
// one MUFU tanh and one FMA.  AETH_TC_SILU selects the arithmetic:
//   0: FP32 tanh and FMA, then rounding to BF16 (one MUFU op per value);
//   1: h rounded to BF16, BF16x2 tanh and BF16x2 FMA (one MUFU op, one FMA
//      and one conversion per pair).
#ifndef AETH_TC_SILU
#define AETH_TC_SILU 0
#endif

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&h);
}

__device__ __forceinline__ float tanh_f32(float x) {
  float t;
  asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(x));
  return t;
}

__device__ __forceinline__ uint32_t tanh_bf16x2(uint32_t x) {
  uint32_t t;
  asm("tanh.approx.bf16x2 %0, %1;" : "=r"(t) : "r"(x));
  return t;
}

// two activations from the raw accumulator words, packed as BF16x2
__device__ __forceinline__ uint32_t silu2(uint32_t a0, uint32_t a1) {
  const float h0 = __uint_as_float(a0), h1 = __uint_as_float(a1);
#if AETH_TC_SILU == 0
  return pack2(fmaf(h0, tanh_f32(h0), h0), fmaf(h1, tanh_f32(h1), h1));
#else
  const uint32_t hh = pack2(h0, h1);
  const uint32_t t = tanh_bf16x2(hh);
  __nv_bfloat162 r = __hfma2(*reinterpret_cast<const __nv_bfloat162*>(&hh),
                             *reinterpret_cast<const __nv_bfloat162*>(&t),
                             *reinterpret_cast<const __nv_bfloat162*>(&hh));
  return *reinterpret_cast<uint32_t*>(&r);
#endif
}

// SiLU of 32 accumulator columns into the A tile (row `row`, columns c0..)
__device__ __forceinline__ void act32(unsigned char* sA, int row, int c0, const uint32_t (&r)[32]) {
#pragma unroll
  for (int h = 0; h < 4; ++h) {
    const uint32_t* v = r + h * 8;
    const uint4 pk = make_uint4(silu2(v[0], v[1]), silu2(v[2], v[3]), silu2(v[4], v[5]), silu2(v[6], v[7]));
    *reinterpret_cast<uint4*>(sA + core_off(row, c0 + h * 8, 128)) = pk;
  }
}

// One warpgroup's state for TPW tiles.  With TPW = 2 the warpgroup owns
// two tiles (ping-pong): while the tensor core runs one tile's layer, the
// warpgroup's threads run the other tile's SiLU epilogue.  Shared-memory
// places are 32-bit offsets from the dynamic shared-memory base.
template <int TPW>
struct WG {
  uint32_t offA[TPW];   // A tiles (layers 2..4)
  uint32_t offX[TPW];   // input tiles (layer 1, bias columns)
  uint32_t bar[TPW];    // one mbarrier per tile (shared address)
  uint32_t tmem;        // first of the warpgroup's TPW x 128 columns, lane 0
  uint32_t lanes;       // this warp's lane quarter in the TMEM address
  // bit t: parity of tile t's next wait; bit 2 + t (issuing thread): tile t
  // has an MMA in flight; bit 4 + t (issuing thread): parity of tile t's
  // completions so far
  uint32_t st;
  int wid;              // thread index in the warpgroup = tile row
  int bar_id;           // named barrier of the warpgroup
};

// Issue layer `layer` of tile t (one thread) and commit it to the tile's
// mbarrier.
template <int TPW>
__device__ __forceinline__ void issue(unsigned char* sm, WG<TPW>& g, int t, int layer) {
  const uint32_t base = smem_u32(sm);
  const uint32_t sA = base + g.offA[t];
  const uint64_t dX = sdesc(base + g.offX[t], 128, 256);
  const uint32_t d = g.tmem + (uint32_t)(t * 128);
  if (layer == 0) {
    mma(d, dX, sdesc(base + OFF_W1, 128, 256), idesc(128, 128), 0);
  } else {
    const uint32_t sB = base + (layer == 1 ? OFF_W2 : (layer == 2 ? OFF_W3 : OFF_W4));
    const uint32_t id = layer == 3 ? idesc(128, 16) : idesc(128, 128);
#pragma unroll
    for (int ks = 0; ks < 8; ++ks)
      mma(d, sdesc(sA + ks * 256, 128, 2048), sdesc(sB + ks * 256, 128, 2048), id, ks > 0);
    if (layer < 3) mma(d, dX, sdesc(base + (layer == 1 ? OFF_BB2 : OFF_BB3), 128, 256), id, 1);
  }
  commit(g.bar[t]);
  g.st |= 4u << t;
}

// this thread's input row of tile t; columns 14, 15 (padding of the 14
// inputs) carry the ones that pick up the biases
template <int TPW>
__device__ __forceinline__ void put_x(unsigned char* sm, const WG<TPW>& g, int t, const float* x) {
  const uint4 lo = make_uint4(pack2(x[0], x[1]), pack2(x[2], x[3]), pack2(x[4], x[5]), pack2(x[6], x[7]));
  const uint4 hi = make_uint4(pack2(x[8], x[9]), pack2(x[10], x[11]), pack2(x[12], x[13]), pack2(1.0f, 1.0f));
  *reinterpret_cast<uint4*>(sm + g.offX[t] + core_off(g.wid, 0, 16)) = lo;
  *reinterpret_cast<uint4*>(sm + g.offX[t] + core_off(g.wid, 8, 16)) = hi;
}

// hidden-layer epilogue of tile t: accumulator -> SiLU -> A tile, the next
// 32 columns loading while the current ones are used
template <int TPW>
__device__ __forceinline__ void epilogue(unsigned char* sm, const WG<TPW>& g, int t) {
  const uint32_t a = g.tmem + (uint32_t)(t * 128) + g.lanes;
  unsigned char* sA = sm + g.offA[t];
  uint32_t ra[32], rb[32];
  tmem_ld32(a, ra);
  tmem_wait32(ra);
  tmem_ld32(a + 32, rb);
  act32(sA, g.wid, 0, ra);
  tmem_wait32(rb);
  tmem_ld32(a + 64, ra);
  act32(sA, g.wid, 32, rb);
  tmem_wait32(ra);
  tmem_ld32(a + 96, rb);
  act32(sA, g.wid, 64, ra);
  tmem_wait32(rb);
  act32(sA, g.wid, 96, rb);
}

// smem tiles written (generic proxy) and TMEM reads done by all 128
// threads before the next MMA; AND-reduces ok over the warpgroup
__device__ __forceinline__ bool wg_handoff(int bar_id, bool ok) {
  fence_async_smem();
  fence_before();
  ok = wg_sync_and(bar_id, ok);
  fence_after();
  return ok;
}

// The network on the warpgroup's TPW tiles of 128 rows: x[t] = this
// thread's 16 inputs of tile t, y[t] its 8 outputs.  With TPW = 2 the two
// tiles alternate on the tensor core (ping-pong).  Returns false, uniformly
// over the warpgroup, if an MMA wait timed out (y undefined).
template <int TPW>
__device__ __forceinline__ bool forward(unsigned char* sm, WG<TPW>& g, const float (*x)[16],
                                        float (*y)[8]) {
#pragma unroll
  for (int t = 0; t < TPW; ++t) put_x(sm, g, t, x[t]);
  if (!wg_handoff(g.bar_id, true)) return false;
  if (g.wid == 0) {
#pragma unroll
    for (int t = 0; t < TPW; ++t) issue(sm, g, t, 0);
  }
  bool ok = true;
#pragma unroll 1
  for (int layer = 0; layer < 4; ++layer) {
#pragma unroll
    for (int t = 0; t < TPW; ++t) {
      const bool got = wait_bar(g.bar[t], (g.st >> t) & 1u);
      g.st ^= 1u << t;
      if (got) g.st = (g.st & ~(4u << t)) ^ (16u << t);
      fence_after();
      ok = ok && got;
      if (got) {
        if (layer < 3) {
          epilogue(sm, g, t);
        } else {
          const float* b4 = reinterpret_cast<const float*>(sm + OFF_B4);
          tmem_ld8(g.tmem + (uint32_t)(t * 128) + g.lanes, y[t]);
#pragma unroll
          for (int q = 0; q < 8; ++q) y[t][q] += b4[q];
        }
      }
      if (layer < 3) {
        ok = wg_handoff(g.bar_id, ok);
        if (!ok) return false;
        if (g.wid == 0) issue(sm, g, t, layer + 1);
      }
    }
  }
  // the next call's input tiles are rewritten: all reads of this call done
  fence_before();
  ok = wg_sync_and(g.bar_id, ok);
  fence_after();
  return ok;
}

// CTA prologue: weights to shared memory, one mbarrier per tile, 128 TMEM
// columns per tile.  Returns this thread's warpgroup state.
template <int NWG, int TPW>
__device__ __forceinline__ WG<TPW> setup(unsigned char* sm, const unsigned char* __restrict__ wimg) {
  constexpr int COLS = NWG * TPW * 128;
  static_assert(COLS == 128 || COLS == 256 || COLS == 512, "TMEM allocation is a power of 2");
  const int tid = threadIdx.x, warp = tid >> 5, wg = tid >> 7;
  {
    const uint4* s = reinterpret_cast<const uint4*>(wimg);
    uint4* d = reinterpret_cast<uint4*>(sm);
    for (int t = tid; t < WBYTES / 16; t += blockDim.x) d[t] = s[t];
  }
  unsigned char* misc = sm + WBYTES + NWG * TPW * WG_BYTES;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(misc + 64);
  if (tid < NWG * TPW) {
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
  WG<TPW> g;
#pragma unroll
  for (int t = 0; t < TPW; ++t) {
    const int slot = wg * TPW + t;
    g.offA[t] = WBYTES + slot * WG_BYTES + WG_A;
    g.offX[t] = WBYTES + slot * WG_BYTES + WG_X;
    g.bar[t] = smem_u32(misc + 8 * slot);
  }
  g.tmem = *tslot + (uint32_t)(wg * TPW * 128);
  g.lanes = (uint32_t)((warp & 3) * 32) << 16;
  g.st = 0;
  g.wid = tid & 127;
  g.bar_id = 1 + wg;
  return g;
}

// CTA epilogue: a warpgroup that timed out raises the status bit and drains
// the MMAs still in flight (bounded waits); then the TMEM columns are
// released.
template <int NWG, int TPW>
__device__ __forceinline__ void teardown(unsigned char* sm, const WG<TPW>& g, bool ok, int* status) {
  if (!ok && g.wid == 0) {
    atomicOr(status, ST_TIMEOUT);
#pragma unroll
    for (int t = 0; t < TPW; ++t)
      if ((g.st >> (2 + t)) & 1u) wait_bar(g.bar[t], (g.st >> (4 + t)) & 1u);
  }
  unsigned char* misc = sm + WBYTES + NWG * TPW * WG_BYTES;
  const uint32_t base = *reinterpret_cast<uint32_t*>(misc + 64);
  fence_before();
  __syncthreads();
  fence_after();
  if ((threadIdx.x >> 5) == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(base), "r"(NWG * TPW * 128)
                 : "memory");
}

// tiles per warpgroup: 1 (four warpgroups, 512 threads, <= 128 registers)
// or 2 (two ping-pong warpgroups, 256 threads); 4 tiles in flight per CTA
// either way (512 TMEM columns, four A/input tile buffers)
#ifndef AETH_TC_TPW
#define AETH_TC_TPW 1
#endif
constexpr int TPW = AETH_TC_TPW;
constexpr int NWG = 4 / TPW;

}  // namespace tc

// X[n][16] -> Y[n][8] (dimensionless rows).
__global__ void __launch_bounds__(tc::NWG * 128, 1)
    k_mlp_tc(const float* __restrict__ X, float* __restrict__ Y, int n,
             const unsigned char* __restrict__ wimg, int* status) {
  using namespace tc;
  extern __shared__ __align__(1024) unsigned char sm[];
  WG<TPW> g = setup<NWG, TPW>(sm, wimg);
  const int wg = threadIdx.x >> 7;
  bool ok = true;
  auto load = [&](int r, float* x) {
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
  };
  auto store = [&](int r, const float* y) {
    if (r < n) {
      float4* dst = reinterpret_cast<float4*>(Y + (long long)r * 8);
      dst[0] = make_float4(y[0], y[1], y[2], y[3]);
      dst[1] = make_float4(y[4], y[5], y[6], y[7]);
    }
  };
  // a warpgroup iteration covers TPW 128-row tiles
  for (long long it = (long long)blockIdx.x * NWG + wg; it * TPW * TM < n; it += (long long)gridDim.x * NWG) {
    float x[TPW][16], y[TPW][8];
#pragma unroll
    for (int t = 0; t < TPW; ++t) load((int)(it * TPW * TM) + t * TM + g.wid, x[t]);
    ok = forward<TPW>(sm, g, x, y);
    if (!ok) break;   // uniform over the warpgroup
#pragma unroll
    for (int t = 0; t < TPW; ++t) store((int)(it * TPW * TM) + t * TM + g.wid, y[t]);
  }
  teardown<NWG, TPW>(sm, g, ok, status);
}

// One face of the learned-flux pass.
template <typename R>
struct FaceIn {
  R wl[7], wr[7], bn;
  long long fc;
  bool valid;
};

// Face source and sink of the learned-flux kernel.  A work unit is 32
// faces, one per lane of a warp; a 128-row tile is 4 work units.
//
// BlockFaces: the faces of direction D of one block in the flux pass: face
// states from the dump arrays (32 faces along x per work unit), fluxes and
// face EMFs into the arrays of the HLLD flux pass.
template <typename R, int D>
struct BlockFaces {
  BlockPtrs<R> P;
  long long nwork;
  int nseg;
  __device__ __forceinline__ void load(long long wk, int lane, FaceIn<R>& f) const {
    const Layout& L = P.L;
    const long long pitch = P.pitch;
    const R* __restrict__ fs = P.fstate;
    f.valid = wk < nwork;
    const long long wkc = f.valid ? wk : 0;
    const int seg = (int)(wkc % nseg);
    const long long row = wkc / nseg;
    const int j = (int)(row % (L.n[1] + 2)) - 1, k = (int)(row / (L.n[1] + 2)) - 1;
    const int i = seg * 32 + lane - 1;
    const int c3[3] = {i, j, k};
    f.valid = f.valid && i <= L.n[0] && c3[D] >= 0;
    f.fc = L.idx(min(i, L.n[0]), j, k);
    if (f.valid) {
#pragma unroll
      for (int q = 0; q < 7; ++q) {
        f.wl[q] = fs[(D * 15 + q) * pitch + f.fc];
        f.wr[q] = fs[(D * 15 + 7 + q) * pitch + f.fc];
      }
      f.bn = fs[(D * 15 + 14) * pitch + f.fc];
    }
  }
  __device__ __forceinline__ void store(const FaceIn<R>& f, const R* F, bool) const {
    constexpr int T1 = (D + 1) % 3, T2 = (D + 2) % 3;
    const long long pitch = P.pitch;
    R* sbp = P.w[0];
    R* fl = sbp + (8 + 5 * D) * pitch + f.fc;
    fl[0] = F[0];
    fl[(1 + D) * pitch] = F[1];
    fl[(1 + T1) * pitch] = F[2];
    fl[(1 + T2) * pitch] = F[3];
    fl[4 * pitch] = F[4];
    R* e = sbp + (23 + 2 * D) * pitch + f.fc;
    e[0] = F[6];
    e[pitch] = -F[5];
  }
};

// FlatFaces: n caller-given faces, st[n][15] = (wl 7, wr 7, bn) in the face
// frame, fluxes into flux[n][7] and the decision into acc[n] (1: network
// accepted, 0: HLLD fallback).
template <typename R>
struct FlatFaces {
  const R* st;
  R* flux;
  int* acc;
  long long n, nwork;
  __device__ __forceinline__ void load(long long wk, int lane, FaceIn<R>& f) const {
    const long long r = wk * 32 + lane;
    f.valid = wk < nwork && r < n;
    f.fc = f.valid ? r : 0;
    if (f.valid) {
      const R* s = st + f.fc * 15;
#pragma unroll
      for (int q = 0; q < 7; ++q) { f.wl[q] = s[q]; f.wr[q] = s[7 + q]; }
      f.bn = s[14];
    }
  }
  __device__ __forceinline__ void store(const FaceIn<R>& f, const R* F, bool accepted) const {
#pragma unroll
    for (int q = 0; q < 7; ++q) flux[f.fc * 7 + q] = F[q];
    acc[f.fc] = accepted ? 1 : 0;
  }
};

// Learned flux of the faces of one face source (the tcgen05 twin of the
// mma.sync flux kernel): face states, network, acceptance test, HLLD on
// rejected faces, fluxes out.  A warpgroup iteration covers TPW tiles.
template <typename R, int TPW, typename IO>
__global__ void __launch_bounds__(512 / TPW, 1)
    k_mlp_flux_tc(IO io, const unsigned char* __restrict__ wimg, R gamma, R tau, int mhd,
                  unsigned long long* fallbacks, int* status) {
  using namespace tc;
  constexpr int NWG = 4 / TPW;
  extern __shared__ __align__(1024) unsigned char sm[];
  WG<TPW> g = setup<NWG, TPW>(sm, wimg);
  const int wg = threadIdx.x >> 7, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long niter = (io.nwork + 4 * TPW - 1) / (4 * TPW);
  unsigned long long fb = 0;
  bool ok = true;
  auto load = [&](long long wk, FaceIn<R>& f, float* x) -> FaceScale {
    io.load(wk, lane, f);
    if (!f.valid) {
#pragma unroll
      for (int q = 0; q < 7; ++q) f.wl[q] = f.wr[q] = R(0);
      f.wl[0] = f.wr[0] = R(1); f.wl[4] = f.wr[4] = R(1);
      f.bn = R(0);
    }
    return mlp_features(f.wl, f.wr, f.bn, gamma, x);
  };
  auto finish = [&](const FaceIn<R>& f, const FaceScale& sc, const float* y) {
    if (!f.valid) return;
    float k7[7];
    mlp_scale_out(sc, (float)gamma, k7);
    R F[7];
    const bool accepted = mlp_compose(gamma, f.wl, f.wr, f.bn, y, k7, tau, mhd != 0, F);
    if (!accepted) {
      hlld(gamma, f.wl, f.wr, f.bn, F);
      ++fb;
    }
    io.store(f, F, accepted);
  };
  for (long long it = (long long)blockIdx.x * NWG + wg; it < niter; it += (long long)gridDim.x * NWG) {
    FaceIn<R> f[TPW];
    FaceScale sc[TPW];
    float x[TPW][16], y[TPW][8];
#pragma unroll
    for (int t = 0; t < TPW; ++t) sc[t] = load((it * TPW + t) * 4 + (warp & 3), f[t], x[t]);
    ok = forward<TPW>(sm, g, x, y);
    if (!ok) break;   // uniform over the warpgroup
#pragma unroll
    for (int t = 0; t < TPW; ++t) finish(f[t], sc[t], y[t]);
  }
  for (int o = 16; o > 0; o >>= 1) fb += __shfl_xor_sync(0xffffffffu, fb, o);
  if (lane == 0 && fb) atomicAdd(fallbacks, fb);
  teardown<NWG, TPW>(sm, g, ok, status);
}

// tiles per warpgroup of the learned-flux kernel: the knob in FP32; 2 for
// FP64 face states (two warpgroups of 256 threads: registers)
template <typename R>
static constexpr int tpw_of() {
  return sizeof(R) == 4 ? tc::TPW : 2;
}

template <typename R>
void mlp_flux_pass_tc(aeth_ctx* c, int block) {
  constexpr int TPW = tpw_of<R>();
  constexpr int NWG = 4 / TPW;
  const BlockPtrs<R> P = block_ptrs<R>(c, block);
  const Layout& L = P.L;
  const long long nseg = (L.n[0] + 2 + 31) / 32;
  const long long niter = (nseg * (L.n[1] + 2) * (L.n[2] + 2) + 4 * TPW - 1) / (4 * TPW);
  // one CTA per SM (shared memory and TMEM columns)
  const int grid = (int)std::max(1LL, std::min((niter + NWG - 1) / NWG, (long long)c->num_sms));
  const R g = (R)c->cfg.gamma;
  const R tau = (R)(c->cfg.mlp_tau > 0 ? c->cfg.mlp_tau : 0.25);
  const int mhd = is_mhd(c);
  const unsigned char* w = (const unsigned char*)c->d_mlp_tc;
  constexpr int SM = tc::smem_bytes(NWG * TPW);
  const long long nwork = nseg * (L.n[1] + 2) * (L.n[2] + 2);
  k_mlp_flux_tc<R, TPW><<<grid, NWG * 128, SM, c->stream>>>(
      BlockFaces<R, 0>{P, nwork, (int)nseg}, w, g, tau, mhd, c->d_fallback, c->d_status);
  k_mlp_flux_tc<R, TPW><<<grid, NWG * 128, SM, c->stream>>>(
      BlockFaces<R, 1>{P, nwork, (int)nseg}, w, g, tau, mhd, c->d_fallback, c->d_status);
  k_mlp_flux_tc<R, TPW><<<grid, NWG * 128, SM, c->stream>>>(
      BlockFaces<R, 2>{P, nwork, (int)nseg}, w, g, tau, mhd, c->d_fallback, c->d_status);
  c->n_launch += 3;
}
template void mlp_flux_pass_tc<float>(aeth_ctx*, int);
template void mlp_flux_pass_tc<double>(aeth_ctx*, int);

// Host: the network's parameters (W_l[out][in], b_l per layer) as the
// shared-memory image above.  Hidden layers are halved (exact in BF16);
// each hidden bias b / 2 is split as hi = bf16(b / 2), lo = bf16(b / 2 - hi).
std::vector<unsigned char> tc_weight_image(const float* params) {
  using namespace tc;
  std::vector<unsigned char> img(WBYTES, 0);
  auto put = [&](int off, int ld_k, int o, int i, float v) {
    const __nv_bfloat16 h = __float2bfloat16(v);
    memcpy(&img[off + core_off(o, i, ld_k)], &h, 2);
  };
  auto split = [&](int off, int o, float b) {
    const __nv_bfloat16 hi = __float2bfloat16(b);
    put(off, 16, o, 14, b);
    put(off, 16, o, 15, b - __bfloat162float(hi));
  };
  const int dims[5] = {14, 128, 128, 128, 7};
  const int woff[4] = {OFF_W1, OFF_W2, OFF_W3, OFF_W4};
  const int ldk[4] = {16, 128, 128, 128};
  const int boff[3] = {OFF_W1, OFF_BB2, OFF_BB3};
  float* b4 = reinterpret_cast<float*>(img.data() + OFF_B4);
  size_t off = 0;
  for (int l = 0; l < 4; ++l) {
    const int nin = dims[l], nout = dims[l + 1];
    const float sc = l < 3 ? 0.5f : 1.0f;
    for (int o = 0; o < nout; ++o)
      for (int i = 0; i < nin; ++i) put(woff[l], ldk[l], o, i, sc * params[off + (size_t)o * nin + i]);
    off += (size_t)nout * nin;
    for (int o = 0; o < nout; ++o) {
      if (l < 3) split(boff[l], o, 0.5f * params[off + o]);
      else b4[o] = params[off + o];
    }
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
  const int sb = smem_bytes(NWG * TPW);
  cudaError_t e = big_smem(k_mlp_tc, sb);
  constexpr int T32 = tpw_of<float>(), T64 = tpw_of<double>();
  if (e == cudaSuccess) e = big_smem(k_mlp_flux_tc<float, T32, BlockFaces<float, 0>>, sb);
  if (e == cudaSuccess) e = big_smem(k_mlp_flux_tc<float, T32, BlockFaces<float, 1>>, sb);
  if (e == cudaSuccess) e = big_smem(k_mlp_flux_tc<float, T32, BlockFaces<float, 2>>, sb);
  if (e == cudaSuccess) e = big_smem(k_mlp_flux_tc<double, T64, BlockFaces<double, 0>>, sb);
  if (e == cudaSuccess) e = big_smem(k_mlp_flux_tc<double, T64, BlockFaces<double, 1>>, sb);
  if (e == cudaSuccess) e = big_smem(k_mlp_flux_tc<double, T64, BlockFaces<double, 2>>, sb);
  if (e == cudaSuccess) e = big_smem(k_mlp_flux_tc<float, T32, FlatFaces<float>>, sb);
  if (e != cudaSuccess) return fail(c, AETH_ERR_CUDA, "tcgen05 network smem attribute: %s", cudaGetErrorString(e));
  return AETH_OK;
}

}  // namespace aeth

namespace aeth {

// One warp waits, through the same bounded wait as the network kernels, on
// an mbarrier that never receives an arrival; the wait gives up after its
// wall-time limit and the kernel reports the time-out in *flag.
__global__ void k_wait_selftest(int* flag) {
  __shared__ __align__(8) uint64_t bar;
  const uint32_t a = tc::smem_u32(&bar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(a) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncwarp();
  const bool got = tc::wait_bar(a, 0u);
  if (threadIdx.x == 0 && !got) atomicOr(flag, ST_TIMEOUT);
}

}  // namespace aeth

extern "C" aeth_status aeth_selftest_wait_timeout(aeth_ctx* c) {
  using namespace aeth;
  if (!c) return AETH_ERR_ARG;
  if (!c->finalized) return fail(c, AETH_ERR_STATE, "call aeth_finalize first");
  int* flag = (int*)(c->arena + c->off_scalars + 512);
  AETH_CK(c, cudaMemsetAsync(flag, 0, sizeof(int), c->stream));
  k_wait_selftest<<<1, 32, 0, c->stream>>>(flag);
  AETH_CK(c, cudaGetLastError());
  c->n_launch += 1;
  int h = 0;
  AETH_CK(c, cudaMemcpyAsync(&h, flag, sizeof h, cudaMemcpyDeviceToHost, c->stream));
  AETH_CK(c, cudaStreamSynchronize(c->stream));
  if (h & ST_TIMEOUT) return fail(c, AETH_ERR_TIMEOUT, "self-test: the bounded wait gave up as designed");
  return AETH_OK;
}

extern "C" aeth_status aeth_mlp_infer_tc(aeth_ctx* c, const float* d_X, float* d_Y, int n) {
  using namespace aeth;
  if (!c || !d_X || !d_Y || n < 0) return AETH_ERR_ARG;
  if (!c->d_mlp_tc) return fail(c, AETH_ERR_STATE, "call aeth_load_mlp first");
  if (((uintptr_t)d_X | (uintptr_t)d_Y) & 15)
    return fail(c, AETH_ERR_ARG, "X and Y must be 16-byte aligned");
  if (n == 0) return AETH_OK;
  const long long iters = ((long long)n + tc::TPW * tc::TM - 1) / (tc::TPW * tc::TM);
  const int grid = (int)std::max(1LL, std::min((iters + tc::NWG - 1) / tc::NWG, (long long)c->num_sms));
  k_mlp_tc<<<grid, tc::NWG * 128, tc::smem_bytes(tc::NWG * tc::TPW), c->stream>>>(
      d_X, d_Y, n, (const unsigned char*)c->d_mlp_tc, c->d_status);
  AETH_CK(c, cudaGetLastError());
  c->n_launch += 1;
  return AETH_OK;
}

extern "C" aeth_status aeth_mlp_face_flux(aeth_ctx* c, const float* d_states, float* d_flux,
                                          int* d_accept, int n) {
  using namespace aeth;
  if (!c || n < 0 || (n > 0 && (!d_states || !d_flux || !d_accept))) return AETH_ERR_ARG;
  if (!c->finalized) return fail(c, AETH_ERR_STATE, "call aeth_finalize first");
  if (!c->d_mlp_tc) return fail(c, AETH_ERR_STATE, "call aeth_load_mlp first");
  if (c->cfg.precision == AETH_FP64 || is_iso(c) || c->cfg.n_dust > 0)
    return fail(c, AETH_ERR_UNSUPPORTED, "the learned flux runs FP32 adiabatic gas only");
  if (n == 0) return AETH_OK;
  constexpr int TPW = tpw_of<float>();
  constexpr int NWG = 4 / TPW;
  const long long nwork = ((long long)n + 31) / 32;
  const long long niter = (nwork + 4 * TPW - 1) / (4 * TPW);
  const int grid = (int)std::max(1LL, std::min((niter + NWG - 1) / NWG, (long long)c->num_sms));
  const float tau = (float)(c->cfg.mlp_tau > 0 ? c->cfg.mlp_tau : 0.25);
  k_mlp_flux_tc<float, TPW><<<grid, NWG * 128, tc::smem_bytes(NWG * TPW), c->stream>>>(
      FlatFaces<float>{d_states, d_flux, d_accept, (long long)n, nwork},
      (const unsigned char*)c->d_mlp_tc, (float)c->cfg.gamma, tau, is_mhd(c) ? 1 : 0,
      c->d_fallback, c->d_status);
  AETH_CK(c, cudaGetLastError());
  c->n_launch += 1;
  return AETH_OK;
}
