// Host runtime of the GB300 MHD library: context, block table, device arena.
#pragma once
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/aether_gb.h"
#include "common.cuh"

namespace aeth {

// Per-block device pointers for one working precision R.
template <typename R>
struct BlockPtrs {
  Layout L;
  Geometry<R> geo;
  R* reg[2][NVAR];     // register A (U^n / u1) and B (stage state / u2)
  R* w[NPRIM];         // primitives (unfused path)
  R* f[3][5];          // hydro fluxes per direction (unfused path)
  R* e[3][2];          // face EMFs per direction: components t1, t2
  R* edge[3];          // corner EMFs by component
  R* dust[2];          // dust registers: [species][4] arrays each (IMEX2P)
  R* dflux;            // dust fluxes: [direction][species][4] arrays
  R* fstate;           // learned flux: face states [direction][wl 7, wr 7, bn]
  const BlockPtrs* tab; // device table of every block of the context (linked
                        // blocks reach their neighbours through it)
  R* ent[2];           // dual energy: entropy S of registers A and B (else null);
                       // its face fluxes use scratch slots 3..5 (fused path)
  long long pitch;     // elements between consecutive arrays of a register
                       // and of the scratch (w, f, e, edge in that order)
};

struct BlockInfo {
  aeth_block_desc desc;
  Layout L;
  long long ncell;        // interior cells
  size_t off_reg[2];      // arena offsets of the two registers (8 arrays)
  size_t off_scratch;     // unfused scratch (w, f, e, edge)
  size_t off_geo;         // geometry tables (R)
  size_t off_dust[2];     // dust registers (n_dust * 4 arrays each)
  size_t off_dflux;       // dust face fluxes [3][n_dust][4] arrays
  size_t off_fstate;      // learned flux: face states [3][15] arrays
  size_t off_ent[2];      // dual energy: entropy array of each register
  size_t geo_len;         // number of R entries in the geometry tables
  int dt_blocks;          // CUDA blocks of this block's dt/diag reductions
  int dt_offset;          // their first slot in the partials array
};

// Pass kinds of the batched launches; each has a prefix sum of tiles per
// mesh block so that one launch covers every block.
enum PassKind : int { PK_FLUX = 0, PK_CELL = 1, PK_FILL0 = 2, PK_FILL1 = 3, PK_FILL2 = 4,
                      PK_ROWS = 5, PK_N = 6 };

// Tile geometry of each pass kind (threads per tile fixed per kind).
// 2-D flux tiles: 128 threads, FLUX_TX x (FLUX_NT / FLUX_TX) by default
// (32 x 4; the autotuner also takes 16 x 8).  Four warps per barrier wait
// less on the slowest warp of a plane than eight: at 256^3, 16 x 8 tiles of
// 128 threads ran 3% faster than 16 x 16 tiles of 256 at the same
// occupancy, for 16% more staged halo.
constexpr int FLUX_TX = 32;
constexpr int FLUX_NT = 128;
// Band tiles (flux tile width 0): whole rows of a block, x from -1 to n_x,
// as many rows as fit FLUX_NT_BAND threads; for blocks with n_x + 2 <= 66 (wider
// blocks keep most lanes of a 2-D tile busy, and the bound keeps the band's
// shared-memory ring within two PPM CTAs per SM).
constexpr int FLUX_BAND_WMAX = 66;
constexpr int FLUX_NT_BAND = 256;
__host__ __device__ constexpr int band_rows(int nx) {
  return FLUX_NT_BAND / (nx + 2) > 1 ? FLUX_NT_BAND / (nx + 2) : 1;
}
// Threads of a flux tile of width tx (0: band tiles).
__host__ __device__ constexpr int flux_threads(int tx) { return tx ? FLUX_NT : FLUX_NT_BAND; }
constexpr int CELL_BX = 32, CELL_BY = 4, CELL_BZ = 2;
constexpr int FILL_TILE = 256;   // ghost cells per tile of the fill pass

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

// Tiles of one block for a pass kind (kchunk: z extent of a flux tile,
// tx: its x width, FLUX_NT / tx its y width; tx = 0: band tiles).
inline int tiles_of(const Layout& L, int kind, int kchunk, int tx = FLUX_TX) {
  const int g = L.g;
  if (kind == PK_FLUX && tx == 0)
    return ceil_div(L.n[1] + 2, band_rows(L.n[0])) * ceil_div(L.n[2] + 2, kchunk);
  if (kind == PK_FLUX)
    return ceil_div(L.n[0] + 2, tx) * ceil_div(L.n[1] + 2, FLUX_NT / tx) *
           ceil_div(L.n[2] + 2, kchunk);
  if (kind == PK_CELL)
    return ceil_div(L.n[0] + 1, CELL_BX) * ceil_div(L.n[1] + 1, CELL_BY) *
           ceil_div(L.n[2] + 1, CELL_BZ);
  if (kind == PK_ROWS) return L.n[1] * L.n[2];
  // ghost slab of axis d, threads mapped linearly over it (FILL_TILE cells
  // per tile)
  const int d = kind - PK_FILL0;
  long long cells = 1;
  for (int e = 0; e < 3; ++e) cells *= e < d ? L.n[e] + 2 * g + 1 : (e == d ? 2 * g + 1 : L.n[e] + 1);
  return (int)((cells + FILL_TILE - 1) / FILL_TILE);
}

}  // namespace aeth

struct aeth_ctx {
  aeth_config cfg;
  std::vector<double> t_stop;
  std::vector<aeth::BlockInfo> blocks;
  cudaStream_t stream = nullptr;
  bool finalized = false;
  bool planned = false;
  int g = 2;                 // ghost width
  size_t elem = 8;           // sizeof working real
  // arena
  char* arena = nullptr;
  size_t arena_bytes = 0;
  bool own_arena = false;
  size_t need = 0;
  size_t off_stage = 0, stage_bytes = 0;   // FP64 host<->device staging
  size_t off_partials = 0;                 // reduction partials (double)
  int n_partials = 0;
  size_t off_scalars = 0;                  // dt, status, counters
  // device scalars (inside the arena)
  double* d_dt = nullptr;        // current step
  double* d_partials = nullptr;
  int* d_status = nullptr;       // latched error bits
  unsigned long long* d_floor = nullptr;
  unsigned long long* d_fallback = nullptr;
  double* d_diag = nullptr;      // 8 doubles
  double* d_stage = nullptr;
  double* d_pack = nullptr;           // device copy of the packed state of every
  size_t pack_doubles = 0;            // block (allocated on first use)
  // CUDA graph of one CFL-driven step (aeth_run)
  cudaGraphExec_t graph = nullptr;
  // MLP parameters (device, bf16/fp32) for the learned flux
  void* d_mlp = nullptr;
  void* d_mlp_tc = nullptr;   // the same network, core-matrix image (tcgen05)
  size_t mlp_n = 0;
  // kernel timing (aeth_profile)
  bool profile = false;
  std::vector<cudaEvent_t> prof_ev;   // pairs: start, stop
  size_t prof_used = 0;               // events recorded so far
  double prof_bytes = 0;              // algorithmic bytes of the timed launches
  long long n_launch = 0;             // kernels launched (all kinds)
  // batched launches: device block table and tile prefix sums
  size_t off_tab = 0, off_prefix = 0;
  // per pass kind, a tile -> (block, local tile) map for contexts of several
  // blocks (cell and fill passes, whose tile counts are fixed at plan time)
  size_t off_tmap[aeth::PK_N] = {};
  int2* d_tmap[aeth::PK_N] = {};
  long long tmap_n[aeth::PK_N] = {};
  void* d_tab = nullptr;              // BlockPtrs<R>[nb]
  std::vector<int3> links;            // block links (below, axis, above)
  size_t off_links = 0;
  int3* d_links = nullptr;            // the same on the device (face mirror pass)
  int* d_prefix = nullptr;            // [PK_N][nb + 1]
  std::vector<int> h_prefix;          // host copy
  int kchunk = 0;                     // z extent of a flux tile (0: choose;
                                      // aeth_autotune times candidates)
  int flux_tx = 32;                   // x width of a flux tile (32 or 16; the y
                                      // width is 128 / flux_tx), or 0: band tiles
  int num_sms = 152;
  int dt_grid = 1;                    // CTAs of the batched reductions
  // error text
  char err[512] = {0};
};

namespace aeth {

enum : int { ST_NONFINITE = 1, ST_FLOOR = 2, ST_TIMEOUT = 4 };

inline aeth_status fail(aeth_ctx* c, aeth_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(c->err, sizeof c->err, fmt, ap);
  va_end(ap);
  return s;
}

#define AETH_CK(ctx, call)                                                   \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess)                                                   \
      return ::aeth::fail((ctx), AETH_ERR_CUDA, "%s failed: %s (%s:%d)", #call, \
                          cudaGetErrorString(e_), __FILE__, __LINE__);        \
  } while (0)

// Device pointers of block b for precision R.
template <typename R>
BlockPtrs<R> block_ptrs(const aeth_ctx* c, int b);

// Kernel sequences (unfused.cu / fused.cu / aux.cu).
aeth_status enqueue_step(aeth_ctx* c, bool cfl_on_device);
aeth_status enqueue_dt(aeth_ctx* c);
aeth_status enqueue_diag(aeth_ctx* c);
// state / dust transfer kernels; io = the FP64 arrays (cons, b1, b2, b3) in
// device-accessible memory: the staging buffer, or the caller's host arrays
// where they are pinned and mapped (read and written over NVLink-C2C)
aeth_status enqueue_load(aeth_ctx* c, int b, double* const* io);
aeth_status enqueue_store(aeth_ctx* c, int b, double* const* io);
aeth_status enqueue_set_dt(aeth_ctx* c, double dt);
aeth_status enqueue_dust_load(aeth_ctx* c, int b, int k, double* io);
aeth_status enqueue_dust_store(aeth_ctx* c, int b, int k, double* io);
aeth_status enqueue_entropy_store(aeth_ctx* c, int b, double* io);
aeth_status build_geometry(aeth_ctx* c);
aeth_status build_tables(aeth_ctx* c);

// Device-side tile -> block lookup (prefix[b] <= t < prefix[b+1]).
__device__ __forceinline__ int find_block(const int* __restrict__ pre, int nb, int t) {
  int lo = 0, hi = nb;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (pre[mid] <= t) lo = mid;
    else hi = mid;
  }
  return lo;
}
// Where a tile's block comes from: the device block table (passes over
// several blocks; binary search of the tile prefix sums), or the kernel's
// parameter space (passes over one block: uniform constant-bank loads).
template <typename R>
struct TableSrc {
  const BlockPtrs<R>* tab;
  const int* pre;
  int nb;
  const int2* map;   // tile -> (block, tile in block), or null: binary search
  __device__ __forceinline__ const BlockPtrs<R>& get(int t, int& loc) const {
    if (map) {
      const int2 e = map[t];
      loc = e.y;
      return tab[e.x];
    }
    const int b = find_block(pre, nb, t);
    loc = t - pre[b];
    return tab[b];
  }
};
template <typename R>
struct ParamSrc {
  BlockPtrs<R> P;
  int base;   // first tile of the block in the pass's numbering
  __device__ __forceinline__ const BlockPtrs<R>& get(int t, int& loc) const {
    loc = t - base;
    return P;
  }
};

inline int prefix_total(const aeth_ctx* c, int kind) {
  const int nb = (int)c->blocks.size();
  return c->h_prefix[kind * (nb + 1) + nb];
}

// Bracket one launch of the dominant kernel with events (aeth_profile).
inline void prof_begin(aeth_ctx* c) {
  if (!c->profile) return;
  if (c->prof_used + 2 > c->prof_ev.size()) {
    for (int q = 0; q < 64; ++q) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      c->prof_ev.push_back(e);
    }
  }
  cudaEventRecord(c->prof_ev[c->prof_used], c->stream);
}
inline void prof_end(aeth_ctx* c, double algo_bytes) {
  if (!c->profile) return;
  cudaEventRecord(c->prof_ev[c->prof_used + 1], c->stream);
  c->prof_used += 2;
  c->prof_bytes += algo_bytes;
}

inline int ghost_width(int recon) {
  return (recon == AETH_RECON_PPM || recon == AETH_RECON_PPM5) ? 3 : (recon == AETH_RECON_PLM ? 2 : 1);
}

inline double cmax_of(int integrator) {
  // IMEX2P: explicit Courant fraction 1/lambda, lambda = 1 + 1/sqrt(2)
  return integrator == AETH_INT_IMEX2P ? 1.0 / (1.0 + 1.0 / 1.4142135623730951) : 1.0;
}

inline bool is_mhd(const aeth_ctx* c) {
  return c->cfg.eos == AETH_EOS_ADIABATIC_MHD || c->cfg.eos == AETH_EOS_ISOTHERMAL_MHD;
}
// isothermal closure p = cs_iso^2 rho (Sec. 2.1): the energy slot is carried
// with zero flux
inline bool is_iso(const aeth_ctx* c) {
  return c->cfg.eos == AETH_EOS_ISOTHERMAL_MHD || c->cfg.eos == AETH_EOS_ISOTHERMAL_HYDRO;
}
// Bytes between consecutive arrays of a block (registers and scratch): the
// array rounded up to 256 bytes.  (Offsetting the array starts against
// each other by extra multiples of 256 bytes was measured to change nothing:
// the DRAM address hash already spreads the ~40 streams of a pass.)
inline size_t array_pitch_bytes(long long cells, int elem) {
  return ((size_t)cells * elem + 255) / 256 * 256;
}

// dual-energy formalism (Sec. 2.8) on
inline bool is_dual(const aeth_ctx* c) { return c->cfg.dual_energy != 0; }

// The flux tile's width may be switched to 16 (FP32 states, the classical
// solvers without dual energy, fused path; the learned flux's state dump
// and the other passes keep the 32-wide tile).
inline bool tile_shape_tunable(const aeth_ctx* c) {
  return c->cfg.precision != AETH_FP64 && !is_dual(c) && c->cfg.riemann != AETH_RIEMANN_MLP &&
         c->cfg.path == AETH_PATH_FUSED;
}

// Band tiles need every block at most FLUX_BAND_WMAX cells wide (with the
// two extra flux columns).
inline bool band_tiles_fit(const aeth_ctx* c) {
  if (!tile_shape_tunable(c)) return false;
  for (const auto& B : c->blocks)
    if (B.L.n[0] + 2 > FLUX_BAND_WMAX) return false;
  return true;
}

// internal solver codes of the unfused face kernel, distinct from every
// AETH_RIEMANN_* value
constexpr int SOLVER_ISO_HLLD = 16;
constexpr int SOLVER_ISO_HLLE = 17;

}  // namespace aeth
