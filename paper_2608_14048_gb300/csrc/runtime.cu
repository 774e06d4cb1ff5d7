// C-ABI entry points of include/aether_gb.h: context, block table, device
// arena, host<->device state transfer, step sequencing and CUDA graphs.
#include <cuda.h>

#include <cmath>
#include <cstring>
#include <new>

#include "runtime.hpp"

using namespace aeth;

namespace aeth {
template <typename R, bool P64> aeth_status step_unfused(aeth_ctx* c);
template <typename R, bool P64> aeth_status step_fused(aeth_ctx* c);
template <typename R, bool P64> aeth_status step_dust(aeth_ctx* c);
size_t geometry_len(const Layout& L);
bool fused_supported(const aeth_ctx* c);

aeth_status enqueue_step(aeth_ctx* c, bool cfl_on_device) {
  if (cfl_on_device) {
    aeth_status s = enqueue_dt(c);
    if (s != AETH_OK) return s;
  }
  const int p = c->cfg.precision;
  if (c->cfg.n_dust > 0) {
    if (p == AETH_FP64) return step_dust<double, false>(c);
    if (p == AETH_FP32) return step_dust<float, false>(c);
    return step_dust<float, true>(c);
  }
  const bool fused = c->cfg.path == AETH_PATH_FUSED && fused_supported(c);
  if (fused) {
    if (p == AETH_FP64) return step_fused<double, false>(c);
    if (p == AETH_FP32) return step_fused<float, false>(c);
    return step_fused<float, true>(c);
  }
  if (p == AETH_FP64) return step_unfused<double, false>(c);
  if (p == AETH_FP32) return step_unfused<float, false>(c);
  return step_unfused<float, true>(c);
}
}  // namespace aeth

static size_t align256(size_t x) { return (x + 255) / 256 * 256; }

extern "C" {

aeth_status aeth_create(const aeth_config* cfg, aeth_ctx** out) {
  if (!cfg || !out) return AETH_ERR_ARG;
  *out = nullptr;
  aeth_ctx* c = new (std::nothrow) aeth_ctx();
  if (!c) return AETH_ERR_OOM;
  c->cfg = *cfg;
  aeth_status bad = AETH_OK;
  if (cfg->eos < AETH_EOS_ADIABATIC_MHD || cfg->eos > AETH_EOS_ISOTHERMAL_HYDRO) bad = AETH_ERR_ARG;
  const bool iso = cfg->eos == AETH_EOS_ISOTHERMAL_MHD || cfg->eos == AETH_EOS_ISOTHERMAL_HYDRO;
  if (!iso && !(cfg->gamma > 1.0)) bad = AETH_ERR_ARG;
  if (iso && !(cfg->cs_iso > 0.0 && cfg->cs_iso < INFINITY)) bad = AETH_ERR_ARG;
  if (cfg->recon < AETH_RECON_DONOR || cfg->recon > AETH_RECON_PPM5) bad = AETH_ERR_ARG;
  if (cfg->riemann < AETH_RIEMANN_HLLD || cfg->riemann > AETH_RIEMANN_LHLLD) bad = AETH_ERR_ARG;
  if (cfg->integrator < AETH_INT_VL2 || cfg->integrator > AETH_INT_RK3) bad = AETH_ERR_ARG;
  if (cfg->precision < AETH_FP64 || cfg->precision > AETH_FP32_SEL64) bad = AETH_ERR_ARG;
  if (!(cfg->cfl > 0.0 && cfg->cfl <= 1.0)) bad = AETH_ERR_ARG;
  if (cfg->path != AETH_PATH_FUSED && cfg->path != AETH_PATH_UNFUSED) bad = AETH_ERR_ARG;
  if (cfg->n_dust < 0 || cfg->n_dust > 32) bad = AETH_ERR_ARG;
  if (cfg->n_dust > 0 && !cfg->t_stop) bad = AETH_ERR_ARG;
  if (cfg->drag_precision < AETH_DRAG_FP64 || cfg->drag_precision > AETH_DRAG_SEL64) bad = AETH_ERR_ARG;
  if (cfg->mlp_engine != AETH_MLP_TCGEN05 && cfg->mlp_engine != AETH_MLP_MMA_SYNC) bad = AETH_ERR_ARG;
  if (bad != AETH_OK) {
    delete c;
    return bad;
  }
  if (cfg->drag_law != AETH_DRAG_LAW_TSTOP && cfg->drag_law != AETH_DRAG_LAW_COEFF) {
    delete c;
    return AETH_ERR_ARG;
  }
  if (cfg->n_dust > 0) {
    // hydro gas (adiabatic or isothermal) under IMEX2P; the per-species
    // FP64 selection needs per-species weights (constant stopping times)
    if ((cfg->eos != AETH_EOS_ADIABATIC_HYDRO && cfg->eos != AETH_EOS_ISOTHERMAL_HYDRO) ||
        cfg->integrator != AETH_INT_IMEX2P ||
        (cfg->drag_law == AETH_DRAG_LAW_COEFF && cfg->drag_precision == AETH_DRAG_SEL64)) {
      delete c;
      return AETH_ERR_UNSUPPORTED;
    }
    c->t_stop.assign(cfg->t_stop, cfg->t_stop + cfg->n_dust);
    for (double t : c->t_stop)
      if (!(t > 0.0)) { delete c; return AETH_ERR_ARG; }
    c->cfg.t_stop = c->t_stop.data();
  } else if (cfg->integrator == AETH_INT_IMEX2P) {
    delete c;
    return AETH_ERR_UNSUPPORTED;
  }
  if (cfg->dual_energy != 0) {
    // dual energy: adiabatic gas, fused path, FP64 or FP32, a classical solver
    const bool ok = !iso && cfg->path == AETH_PATH_FUSED &&
                    (cfg->precision == AETH_FP64 || cfg->precision == AETH_FP32) &&
                    cfg->riemann != AETH_RIEMANN_MLP && cfg->n_dust == 0;
    if (!ok) {
      delete c;
      return AETH_ERR_UNSUPPORTED;
    }
    if (!(c->cfg.alpha_switch > 0.0)) c->cfg.alpha_switch = 1e-3;
    if (!(c->cfg.alpha_sync > 0.0)) c->cfg.alpha_sync = 1e-1;
  }
  if (iso && cfg->riemann == AETH_RIEMANN_LHLLD) {
    delete c;
    return AETH_ERR_UNSUPPORTED;   // isothermal solvers: HLLD and HLLE
  }
  if (cfg->riemann == AETH_RIEMANN_MLP && (cfg->precision == AETH_FP64 || cfg->n_dust > 0 || iso)) {
    delete c;
    return AETH_ERR_UNSUPPORTED;   // the learned flux runs with FP32 adiabatic states, gas only
  }
  if (cfg->precision == AETH_FP32_SEL64 && !(c->cfg.p64_ratio > 0.0)) c->cfg.p64_ratio = 4.0;
  if (cfg->drag_precision == AETH_DRAG_SEL64 && !(c->cfg.drag_ratio > 0.0)) c->cfg.drag_ratio = 1.0;
  c->elem = cfg->precision == AETH_FP64 ? 8 : 4;
  c->g = ghost_width(cfg->recon);
  *out = c;
  return AETH_OK;
}

aeth_status aeth_bind_stream(aeth_ctx* c, void* stream) {
  if (!c) return AETH_ERR_ARG;
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  c->stream = (cudaStream_t)stream;
  return AETH_OK;
}

aeth_status aeth_bind_arena(aeth_ctx* c, void* p, size_t bytes) {
  if (!c || !p) return AETH_ERR_ARG;
  if (c->finalized) return fail(c, AETH_ERR_STATE, "arena must be bound before aeth_finalize");
  if (((uintptr_t)p) % 256 != 0) return fail(c, AETH_ERR_ARG, "arena must be 256-byte aligned");
  c->arena = (char*)p;
  c->arena_bytes = bytes;
  c->own_arena = false;
  return AETH_OK;
}

aeth_status aeth_add_block(aeth_ctx* c, const aeth_block_desc* d, int* id) {
  if (!c || !d) return AETH_ERR_ARG;
  if (c->finalized || c->planned) return fail(c, AETH_ERR_STATE, "blocks must be added before plan/finalize");
  if (d->nx < 1 || d->ny < 1 || d->nz < 1) return fail(c, AETH_ERR_ARG, "block sizes must be >= 1");
  if ((long long)d->nx * d->ny * d->nz > (1ll << 31))
    return fail(c, AETH_ERR_ARG, "block of %lld cells exceeds 2^31", (long long)d->nx * d->ny * d->nz);
  if (!(d->x1max > d->x1min && d->x2max > d->x2min && d->x3max > d->x3min))
    return fail(c, AETH_ERR_ARG, "block extents must be increasing");
  if (d->coord != AETH_COORD_CART && d->coord != AETH_COORD_SPH) return fail(c, AETH_ERR_ARG, "bad coord");
  for (int q = 0; q < 3; ++q)
    if (d->bc[q] != AETH_BC_PERIODIC && d->bc[q] != AETH_BC_OUTFLOW) return fail(c, AETH_ERR_ARG, "bad bc");
  const int g = c->g;
  const int nn[3] = {d->nx, d->ny, d->nz};
  for (int q = 0; q < 3; ++q)
    if (d->bc[q] == AETH_BC_PERIODIC && nn[q] < g && nn[q] != 1)
      return fail(c, AETH_ERR_ARG, "periodic axis %d needs n >= ghost width %d (or n == 1)", q, g);
  if (d->coord == AETH_COORD_SPH && c->cfg.integrator == AETH_INT_RK3)
    return fail(c, AETH_ERR_UNSUPPORTED, "SSP-RK3 runs on Cartesian blocks only");
  if (d->coord == AETH_COORD_SPH && c->cfg.n_dust > 0)
    return fail(c, AETH_ERR_UNSUPPORTED, "dust runs support Cartesian blocks only");
  if (d->coord == AETH_COORD_SPH) {
    if (!(d->x1min - g * (d->x1max - d->x1min) / d->nx > 0.0))
      return fail(c, AETH_ERR_ARG, "spherical block: r (incl. ghosts) must stay > 0");
    const double dth = (d->x2max - d->x2min) / d->ny;
    if (!(d->x2min - g * dth > 0.0 && d->x2max + g * dth < M_PI))
      return fail(c, AETH_ERR_ARG, "spherical block: theta (incl. ghosts) must avoid the axis");
  }
  BlockInfo B{};
  B.desc = *d;
  Layout& L = B.L;
  L.n[0] = d->nx; L.n[1] = d->ny; L.n[2] = d->nz;
  L.g = g;
  for (int q = 0; q < 3; ++q) L.bc[q] = d->bc[q];
  L.coord = d->coord;
  L.self = (int)c->blocks.size();
  for (int q = 0; q < 3; ++q) L.lnk[q][0] = L.lnk[q][1] = -1;
  L.p64_ratio = c->cfg.precision == AETH_FP32_SEL64 ? (float)c->cfg.p64_ratio : 0.0f;
  L.sx = ((long long)OX + d->nx + g + 1 + 3) / 4 * 4;
  L.sy = d->ny + 2 * g + 1;
  L.sz = d->nz + 2 * g + 1;
  B.ncell = (long long)d->nx * d->ny * d->nz;
  c->blocks.push_back(B);
  if (id) *id = (int)c->blocks.size() - 1;
  return AETH_OK;
}

aeth_status aeth_link_blocks(aeth_ctx* c, int lo, int axis, int hi) {
  if (!c) return AETH_ERR_ARG;
  if (c->finalized || c->planned) return fail(c, AETH_ERR_STATE, "links must be set before plan/finalize");
  const int nb = (int)c->blocks.size();
  if (lo < 0 || lo >= nb || hi < 0 || hi >= nb || axis < 0 || axis > 2)
    return fail(c, AETH_ERR_ARG, "bad block index or axis");
  Layout& A = c->blocks[lo].L;
  Layout& B = c->blocks[hi].L;
  if (A.lnk[axis][1] >= 0 || B.lnk[axis][0] >= 0)
    return fail(c, AETH_ERR_ARG, "side already linked");
  if (A.coord != AETH_COORD_CART || B.coord != AETH_COORD_CART)
    return fail(c, AETH_ERR_UNSUPPORTED, "linked blocks must be Cartesian");
  for (int e = 0; e < 3; ++e)
    if (e != axis && A.n[e] != B.n[e])
      return fail(c, AETH_ERR_ARG, "linked blocks differ across the shared face (axis %d)", e);
  if (A.n[axis] < c->g || B.n[axis] < c->g)
    return fail(c, AETH_ERR_ARG, "linked blocks need >= %d cells along the link axis", c->g);
  {
    // one uniform grid: equal cell widths on every axis and coinciding
    // extents across the shared face
    const aeth_block_desc& a = c->blocks[lo].desc;
    const aeth_block_desc& b = c->blocks[hi].desc;
    const double alo[3] = {a.x1min, a.x2min, a.x3min}, ahi[3] = {a.x1max, a.x2max, a.x3max};
    const double blo[3] = {b.x1min, b.x2min, b.x3min}, bhi[3] = {b.x1max, b.x2max, b.x3max};
    for (int e = 0; e < 3; ++e) {
      const double da = (ahi[e] - alo[e]) / A.n[e], db = (bhi[e] - blo[e]) / B.n[e];
      const double tol = 1e-9 * std::max(std::fabs(da), std::fabs(db));
      if (std::fabs(da - db) > tol)
        return fail(c, AETH_ERR_ARG, "linked blocks differ in cell width along axis %d", e);
      if (e != axis && (std::fabs(alo[e] - blo[e]) > tol || std::fabs(ahi[e] - bhi[e]) > tol))
        return fail(c, AETH_ERR_ARG, "linked blocks are not aligned across the face (axis %d)", e);
    }
  }
  if (c->cfg.path != AETH_PATH_FUSED || c->cfg.n_dust > 0)
    return fail(c, AETH_ERR_UNSUPPORTED, "linked blocks run on the fused gas path");
  A.lnk[axis][1] = hi;
  B.lnk[axis][0] = lo;
  c->links.push_back(make_int3(lo, axis, hi));
  return AETH_OK;
}

aeth_status aeth_plan(aeth_ctx* c, size_t* bytes) {
  if (!c) return AETH_ERR_ARG;
  if (c->blocks.empty()) return fail(c, AETH_ERR_STATE, "no blocks");
  size_t off = 0;
  size_t max_stage = 0;
  int npart = 0;
  for (auto& B : c->blocks) {
    const long long sz = B.L.size();
    const size_t arr = array_pitch_bytes(sz, c->elem);
    for (int r = 0; r < 2; ++r) {
      B.off_reg[r] = off;
      off += NVAR * arr;
    }
    // stage scratch: primitives (unfused) or reference EMFs (fused) in the
    // first slots, then face fluxes, face EMFs and corner EMFs
    B.off_scratch = off;
    off += (NPRIM + 15 + 6 + 3) * arr;
    if (c->cfg.n_dust > 0) {
      for (int r = 0; r < 2; ++r) {
        B.off_dust[r] = off;
        off += align256((size_t)4 * c->cfg.n_dust * sz * c->elem);
      }
      B.off_dflux = off;
      off += align256((size_t)12 * c->cfg.n_dust * sz * c->elem);
    }
    if (c->cfg.riemann == AETH_RIEMANN_MLP) {
      B.off_fstate = off;
      off += 45 * arr;
    }
    if (is_dual(c)) {
      for (int r = 0; r < 2; ++r) {
        B.off_ent[r] = off;
        off += arr;
      }
    }
    B.geo_len = geometry_len(B.L);
    B.off_geo = off;
    off += align256(B.geo_len * c->elem);
    const long long nx = B.desc.nx, ny = B.desc.ny, nz = B.desc.nz;
    size_t st = (size_t)(5 * nx * ny * nz + nz * ny * (nx + 1) + nz * (ny + 1) * nx + (nz + 1) * ny * nx);
    if (c->cfg.n_dust > 0) st = std::max(st, (size_t)(4 * nx * ny * nz));
    max_stage = std::max(max_stage, st * sizeof(double));
    npart += B.desc.ny * B.desc.nz;   // x-rows of this block
  }
  // batched reductions: at most 8192 CTAs, each reducing whole x-rows
  c->dt_grid = std::max(1, std::min(npart, 8192));
  npart = c->dt_grid;
  // device block table and tile prefix sums of the batched passes
  const int nb = (int)c->blocks.size();
  c->off_tab = off;
  off += align256((size_t)nb * sizeof(BlockPtrs<double>));
  c->off_links = off;
  off += align256(std::max<size_t>(1, c->links.size()) * sizeof(int3));
  c->off_prefix = off;
  off += align256((size_t)PK_N * (nb + 1) * sizeof(int));
  for (int kind = 0; kind < PK_N; ++kind) {
    c->tmap_n[kind] = 0;
    if (nb < 2 || !(kind == PK_CELL || (kind >= PK_FILL0 && kind <= PK_FILL2))) continue;
    long long tiles = 0;
    for (const auto& B : c->blocks) tiles += tiles_of(B.L, kind, 0);
    c->off_tmap[kind] = off;
    c->tmap_n[kind] = tiles;
    off += align256((size_t)tiles * sizeof(int2));
  }
  c->off_stage = off;
  c->stage_bytes = align256(max_stage);
  off += c->stage_bytes;
  c->off_partials = off;
  c->n_partials = npart;
  off += align256((size_t)6 * npart * sizeof(double));
  c->off_scalars = off;
  off += 4096;
  c->need = off;
  c->planned = true;
  if (bytes) *bytes = off;
  return AETH_OK;
}

aeth_status aeth_finalize(aeth_ctx* c, size_t* bytes) {
  if (!c) return AETH_ERR_ARG;
  if (c->finalized) return fail(c, AETH_ERR_STATE, "already finalized");
  aeth_status s = aeth_plan(c, bytes);
  if (s != AETH_OK) return s;
  if (c->arena) {
    if (c->arena_bytes < c->need)
      return fail(c, AETH_ERR_ARG, "bound arena has %zu bytes, %zu needed", c->arena_bytes, c->need);
  } else {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, c->need);
    if (e != cudaSuccess)
      return fail(c, AETH_ERR_OOM, "cudaMalloc(%zu) failed: %s", c->need, cudaGetErrorString(e));
    c->arena = (char*)p;
    c->arena_bytes = c->need;
    c->own_arena = true;
  }
  AETH_CK(c, cudaMemsetAsync(c->arena, 0, c->need, c->stream));
  c->d_stage = (double*)(c->arena + c->off_stage);
  c->d_partials = (double*)(c->arena + c->off_partials);
  char* sc = c->arena + c->off_scalars;
  c->d_dt = (double*)sc;
  c->d_diag = (double*)(sc + 64);
  c->d_status = (int*)(sc + 256);
  c->d_floor = (unsigned long long*)(sc + 320);
  c->d_fallback = (unsigned long long*)(sc + 384);
  s = build_geometry(c);
  if (s != AETH_OK) return s;
  int dev = 0;
  AETH_CK(c, cudaGetDevice(&dev));
  AETH_CK(c, cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev));
  c->d_tab = c->arena + c->off_tab;
  c->d_prefix = (int*)(c->arena + c->off_prefix);
  c->d_links = (int3*)(c->arena + c->off_links);
  if (!c->links.empty())
    AETH_CK(c, cudaMemcpyAsync(c->d_links, c->links.data(), c->links.size() * sizeof(int3),
                               cudaMemcpyHostToDevice, c->stream));
  for (int kind = 0; kind < PK_N; ++kind)
    c->d_tmap[kind] = c->tmap_n[kind] > 0 ? (int2*)(c->arena + c->off_tmap[kind]) : nullptr;
  s = build_tables(c);
  if (s != AETH_OK) return s;
  AETH_CK(c, cudaStreamSynchronize(c->stream));
  c->finalized = true;
  return AETH_OK;
}

static aeth_status check_block(aeth_ctx* c, int b) {
  if (!c) return AETH_ERR_ARG;
  if (!c->finalized) return fail(c, AETH_ERR_STATE, "call aeth_finalize first");
  if (b < 0 || b >= (int)c->blocks.size()) return fail(c, AETH_ERR_ARG, "block %d out of range", b);
  return AETH_OK;
}

static aeth_status read_status(aeth_ctx* c) {
  int st = 0;
  AETH_CK(c, cudaMemcpyAsync(&st, c->d_status, sizeof st, cudaMemcpyDeviceToHost, c->stream));
  AETH_CK(c, cudaStreamSynchronize(c->stream));
  if (st & ST_NONFINITE) return fail(c, AETH_ERR_NONFINITE, "non-finite value in the state");
  if (st & ST_TIMEOUT) return fail(c, AETH_ERR_TIMEOUT, "a bounded device wait gave up");
  if (st & ST_FLOOR) return fail(c, AETH_ERR_FLOOR, "floor applied with strict_floors set");
  return AETH_OK;
}

// Device address of a caller's host array of `bytes`, or null.  Only memory
// the CUDA runtime has pinned and mapped (cudaHostAlloc, cudaHostRegister)
// qualifies, and only when its allocation range covers the whole array:
// the transfer kernels then read or write it directly over NVLink-C2C.
// Anything else (pageable memory, a failed query) goes through the staging
// buffer and cudaMemcpy.
static void* mapped_host(const void* p, size_t bytes) {
  if (!p || bytes == 0) return nullptr;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (at.type != cudaMemoryTypeHost || !at.devicePointer) return nullptr;
  using GetAttr = CUresult (*)(void*, CUpointer_attribute, CUdeviceptr);
  static GetAttr get = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuPointerGetAttribute", &f, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return (GetAttr) nullptr;
    }
    return (GetAttr)f;
  }();
  if (!get) return nullptr;
  const CUdeviceptr dp = (CUdeviceptr)(uintptr_t)at.devicePointer;
  CUdeviceptr start = 0;
  size_t size = 0;
  if (get(&start, CU_POINTER_ATTRIBUTE_RANGE_START_ADDR, dp) != CUDA_SUCCESS) return nullptr;
  if (get(&size, CU_POINTER_ATTRIBUTE_RANGE_SIZE, dp) != CUDA_SUCCESS) return nullptr;
  if (dp < start || dp + bytes > start + size) return nullptr;
  return at.devicePointer;
}

aeth_status aeth_set_state(aeth_ctx* c, int b, const double* cons, const double* b1,
                           const double* b2, const double* b3) {
  aeth_status s = check_block(c, b);
  if (s != AETH_OK) return s;
  if (!cons) return fail(c, AETH_ERR_ARG, "cons is NULL");
  const auto& B = c->blocks[b];
  const long long nx = B.desc.nx, ny = B.desc.ny, nz = B.desc.nz, nc = nx * ny * nz;
  const bool mhd = is_mhd(c);
  if (mhd && (!b1 || !b2 || !b3)) return fail(c, AETH_ERR_ARG, "face fields are NULL");
  const size_t bytes[4] = {5 * nc * sizeof(double), nz * ny * (nx + 1) * sizeof(double),
                           nz * (ny + 1) * nx * sizeof(double), (nz + 1) * ny * nx * sizeof(double)};
  const double* host[4] = {cons, b1, b2, b3};
  double* io[4] = {nullptr, nullptr, nullptr, nullptr};
  bool direct = true;
  for (int q = 0; q < (mhd ? 4 : 1); ++q) {
    io[q] = (double*)mapped_host(host[q], bytes[q]);
    direct = direct && io[q];
  }
  if (!direct) {
    double* d = c->d_stage;
    for (int q = 0; q < (mhd ? 4 : 1); ++q) {
      io[q] = d;
      AETH_CK(c, cudaMemcpyAsync(d, host[q], bytes[q], cudaMemcpyHostToDevice, c->stream));
      d += bytes[q] / sizeof(double);
    }
  }
  s = enqueue_load(c, b, io);
  if (s != AETH_OK) return s;
  AETH_CK(c, cudaStreamSynchronize(c->stream));
  return AETH_OK;
}

// true when the caller's host array of `bytes` is page-locked memory the
// copy engines can read or write asynchronously
static bool page_locked(const void* p, size_t bytes) {
  if (!p || bytes == 0) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeHost;
}

aeth_status aeth_set_state_async(aeth_ctx* c, int b, const double* cons, const double* b1,
                                 const double* b2, const double* b3) {
  aeth_status s = check_block(c, b);
  if (s != AETH_OK) return s;
  if (!cons) return fail(c, AETH_ERR_ARG, "cons is NULL");
  const auto& B = c->blocks[b];
  const long long nx = B.desc.nx, ny = B.desc.ny, nz = B.desc.nz, nc = nx * ny * nz;
  const bool mhd = is_mhd(c);
  if (mhd && (!b1 || !b2 || !b3)) return fail(c, AETH_ERR_ARG, "face fields are NULL");
  const size_t bytes[4] = {5 * nc * sizeof(double), nz * ny * (nx + 1) * sizeof(double),
                           nz * (ny + 1) * nx * sizeof(double), (nz + 1) * ny * nx * sizeof(double)};
  const double* host[4] = {cons, b1, b2, b3};
  double* io[4] = {nullptr, nullptr, nullptr, nullptr};
  double* d = c->d_stage;
  for (int q = 0; q < (mhd ? 4 : 1); ++q) {
    if (!page_locked(host[q], bytes[q]))
      return fail(c, AETH_ERR_ARG, "array %d is not page-locked host memory", q);
    io[q] = d;
    AETH_CK(c, cudaMemcpyAsync(d, host[q], bytes[q], cudaMemcpyHostToDevice, c->stream));
    d += bytes[q] / sizeof(double);
  }
  return enqueue_load(c, b, io);
}

aeth_status aeth_get_state_async(aeth_ctx* c, int b, double* cons, double* b1, double* b2,
                                 double* b3) {
  aeth_status s = check_block(c, b);
  if (s != AETH_OK) return s;
  if (!cons) return fail(c, AETH_ERR_ARG, "cons is NULL");
  const auto& B = c->blocks[b];
  const long long nx = B.desc.nx, ny = B.desc.ny, nz = B.desc.nz, nc = nx * ny * nz;
  const bool faces = is_mhd(c) && b1 && b2 && b3;
  const size_t bytes[4] = {5 * nc * sizeof(double), nz * ny * (nx + 1) * sizeof(double),
                           nz * (ny + 1) * nx * sizeof(double), (nz + 1) * ny * nx * sizeof(double)};
  double* host[4] = {cons, b1, b2, b3};
  double* io[4] = {nullptr, nullptr, nullptr, nullptr};
  double* d = c->d_stage;
  for (int q = 0; q < 4; ++q) {
    if (q < (faces ? 4 : 1) && !page_locked(host[q], bytes[q]))
      return fail(c, AETH_ERR_ARG, "array %d is not page-locked host memory", q);
    io[q] = d;
    d += bytes[q] / sizeof(double);
  }
  s = enqueue_store(c, b, io);
  if (s != AETH_OK) return s;
  for (int q = 0; q < (faces ? 4 : 1); ++q)
    AETH_CK(c, cudaMemcpyAsync(host[q], io[q], bytes[q], cudaMemcpyDeviceToHost, c->stream));
  return AETH_OK;
}

// Doubles of one block's packed state: cons [5][nz][ny][nx], then in MHD
// b1 [nz][ny][nx+1], b2 [nz][ny+1][nx], b3 [nz+1][ny][nx], then with dust
// every species' [4][nz][ny][nx] (part[4]: all species).
static size_t packed_doubles(const aeth_ctx* c, int b, size_t part[5]) {
  const auto& B = c->blocks[b];
  const size_t nx = B.desc.nx, ny = B.desc.ny, nz = B.desc.nz;
  part[0] = 5 * nx * ny * nz;
  part[1] = is_mhd(c) ? nz * ny * (nx + 1) : 0;
  part[2] = is_mhd(c) ? nz * (ny + 1) * nx : 0;
  part[3] = is_mhd(c) ? (nz + 1) * ny * nx : 0;
  part[4] = (size_t)c->cfg.n_dust * 4 * nx * ny * nz;
  return part[0] + part[1] + part[2] + part[3] + part[4];
}

aeth_status aeth_state_doubles(aeth_ctx* c, size_t* n) {
  if (!c || !n) return AETH_ERR_ARG;
  if (!c->finalized) return fail(c, AETH_ERR_STATE, "call aeth_finalize first");
  size_t t = 0, part[5];
  for (int b = 0; b < (int)c->blocks.size(); ++b) t += packed_doubles(c, b, part);
  *n = t;
  return AETH_OK;
}

static aeth_status pack_buffer(aeth_ctx* c, const void* host, size_t* total) {
  aeth_status s = aeth_state_doubles(c, total);
  if (s != AETH_OK) return s;
  if (!page_locked(host, *total * sizeof(double)))
    return fail(c, AETH_ERR_ARG, "the packed array is not page-locked host memory");
  if (!c->d_pack) {
    if (cudaMalloc(&c->d_pack, *total * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      c->d_pack = nullptr;
      return fail(c, AETH_ERR_OOM, "packed staging buffer (%zu bytes)", *total * sizeof(double));
    }
    c->pack_doubles = *total;
  }
  return AETH_OK;
}

aeth_status aeth_set_state_all_async(aeth_ctx* c, const double* packed) {
  if (!c || !packed) return AETH_ERR_ARG;
  size_t total = 0;
  aeth_status s = pack_buffer(c, packed, &total);
  if (s != AETH_OK) return s;
  AETH_CK(c, cudaMemcpyAsync(c->d_pack, packed, total * sizeof(double), cudaMemcpyHostToDevice,
                             c->stream));
  double* d = c->d_pack;
  for (int b = 0; b < (int)c->blocks.size(); ++b) {
    size_t part[5];
    const size_t n = packed_doubles(c, b, part);
    double* io[4] = {d, d + part[0], d + part[0] + part[1], d + part[0] + part[1] + part[2]};
    s = enqueue_load(c, b, io);
    if (s != AETH_OK) return s;
    double* dd = d + part[0] + part[1] + part[2] + part[3];
    for (int k = 0; k < c->cfg.n_dust; ++k) {
      s = enqueue_dust_load(c, b, k, dd + (size_t)k * (part[4] / c->cfg.n_dust));
      if (s != AETH_OK) return s;
    }
    d += n;
  }
  return AETH_OK;
}

aeth_status aeth_get_state_all_async(aeth_ctx* c, double* packed) {
  if (!c || !packed) return AETH_ERR_ARG;
  size_t total = 0;
  aeth_status s = pack_buffer(c, packed, &total);
  if (s != AETH_OK) return s;
  double* d = c->d_pack;
  for (int b = 0; b < (int)c->blocks.size(); ++b) {
    size_t part[5];
    const size_t n = packed_doubles(c, b, part);
    double* io[4] = {d, d + part[0], d + part[0] + part[1], d + part[0] + part[1] + part[2]};
    s = enqueue_store(c, b, io);
    if (s != AETH_OK) return s;
    double* dd = d + part[0] + part[1] + part[2] + part[3];
    for (int k = 0; k < c->cfg.n_dust; ++k) {
      s = enqueue_dust_store(c, b, k, dd + (size_t)k * (part[4] / c->cfg.n_dust));
      if (s != AETH_OK) return s;
    }
    d += n;
  }
  AETH_CK(c, cudaMemcpyAsync(packed, c->d_pack, total * sizeof(double), cudaMemcpyDeviceToHost,
                             c->stream));
  return AETH_OK;
}

aeth_status aeth_get_state(aeth_ctx* c, int b, double* cons, double* b1, double* b2, double* b3) {
  aeth_status s = check_block(c, b);
  if (s != AETH_OK) return s;
  if (!cons) return fail(c, AETH_ERR_ARG, "cons is NULL");
  const auto& B = c->blocks[b];
  const long long nx = B.desc.nx, ny = B.desc.ny, nz = B.desc.nz, nc = nx * ny * nz;
  const bool faces = is_mhd(c) && b1 && b2 && b3;
  const size_t bytes[4] = {5 * nc * sizeof(double), nz * ny * (nx + 1) * sizeof(double),
                           nz * (ny + 1) * nx * sizeof(double), (nz + 1) * ny * nx * sizeof(double)};
  double* host[4] = {cons, b1, b2, b3};
  double* io[4] = {nullptr, nullptr, nullptr, nullptr};
  bool direct = true;
  for (int q = 0; q < (faces ? 4 : 1); ++q) {
    io[q] = (double*)mapped_host(host[q], bytes[q]);
    direct = direct && io[q];
  }
  if (!direct) {
    double* d = c->d_stage;
    for (int q = 0; q < 4; ++q) {
      io[q] = d;
      d += bytes[q] / sizeof(double);
    }
  } else if (!faces) {
    // the store kernel writes the face fields of an MHD state: into staging
    double* d = c->d_stage;
    for (int q = 1; q < 4; ++q) {
      io[q] = d;
      d += bytes[q] / sizeof(double);
    }
  }
  s = enqueue_store(c, b, io);
  if (s != AETH_OK) return s;
  if (!direct) {
    AETH_CK(c, cudaMemcpyAsync(cons, io[0], bytes[0], cudaMemcpyDeviceToHost, c->stream));
    if (faces)
      for (int q = 1; q < 4; ++q)
        AETH_CK(c, cudaMemcpyAsync(host[q], io[q], bytes[q], cudaMemcpyDeviceToHost, c->stream));
  }
  AETH_CK(c, cudaStreamSynchronize(c->stream));
  return read_status(c);
}

aeth_status aeth_get_entropy(aeth_ctx* c, int b, double* S) {
  aeth_status s = check_block(c, b);
  if (s != AETH_OK) return s;
  if (!S) return fail(c, AETH_ERR_ARG, "S is NULL");
  if (!is_dual(c)) return fail(c, AETH_ERR_STATE, "dual energy is off");
  const size_t bytes = c->blocks[b].ncell * sizeof(double);
  double* mapped = (double*)mapped_host(S, bytes);
  s = enqueue_entropy_store(c, b, mapped ? mapped : c->d_stage);
  if (s != AETH_OK) return s;
  if (!mapped) AETH_CK(c, cudaMemcpyAsync(S, c->d_stage, bytes, cudaMemcpyDeviceToHost, c->stream));
  AETH_CK(c, cudaStreamSynchronize(c->stream));
  return read_status(c);
}

aeth_status aeth_set_dust(aeth_ctx* c, int b, int k, const double* rm) {
  aeth_status s = check_block(c, b);
  if (s != AETH_OK) return s;
  if (k < 0 || k >= c->cfg.n_dust || !rm) return fail(c, AETH_ERR_ARG, "bad dust species or NULL");
  const auto& B = c->blocks[b];
  const size_t bytes = 4 * B.ncell * sizeof(double);
  double* io = (double*)mapped_host(rm, bytes);
  if (!io) {
    io = c->d_stage;
    AETH_CK(c, cudaMemcpyAsync(io, rm, bytes, cudaMemcpyHostToDevice, c->stream));
  }
  s = enqueue_dust_load(c, b, k, io);
  if (s != AETH_OK) return s;
  AETH_CK(c, cudaStreamSynchronize(c->stream));
  return AETH_OK;
}

aeth_status aeth_get_dust(aeth_ctx* c, int b, int k, double* rm) {
  aeth_status s = check_block(c, b);
  if (s != AETH_OK) return s;
  if (k < 0 || k >= c->cfg.n_dust || !rm) return fail(c, AETH_ERR_ARG, "bad dust species or NULL");
  const auto& B = c->blocks[b];
  const size_t bytes = 4 * B.ncell * sizeof(double);
  double* mapped = (double*)mapped_host(rm, bytes);
  s = enqueue_dust_store(c, b, k, mapped ? mapped : c->d_stage);
  if (s != AETH_OK) return s;
  if (!mapped)
    AETH_CK(c, cudaMemcpyAsync(rm, c->d_stage, bytes, cudaMemcpyDeviceToHost, c->stream));
  AETH_CK(c, cudaStreamSynchronize(c->stream));
  return read_status(c);
}

aeth_status aeth_compute_dt(aeth_ctx* c, double* dt) {
  if (!c || !dt) return AETH_ERR_ARG;
  if (!c->finalized) return fail(c, AETH_ERR_STATE, "call aeth_finalize first");
  aeth_status s = enqueue_dt(c);
  if (s != AETH_OK) return s;
  AETH_CK(c, cudaMemcpyAsync(dt, c->d_dt, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  AETH_CK(c, cudaStreamSynchronize(c->stream));
  return read_status(c);
}

aeth_status aeth_step(aeth_ctx* c, double dt) {
  if (!c) return AETH_ERR_ARG;
  if (!c->finalized) return fail(c, AETH_ERR_STATE, "call aeth_finalize first");
  if (!(dt >= 0.0) || !std::isfinite(dt)) return fail(c, AETH_ERR_ARG, "dt must be finite and >= 0");
  if (dt > 0.0) {
    aeth_status s = enqueue_set_dt(c, dt);
    if (s != AETH_OK) return s;
  }
  return enqueue_step(c, false);
}

aeth_status aeth_run(aeth_ctx* c, int nsteps) {
  if (!c) return AETH_ERR_ARG;
  if (!c->finalized) return fail(c, AETH_ERR_STATE, "call aeth_finalize first");
  if (nsteps < 0) return fail(c, AETH_ERR_ARG, "nsteps < 0");
  if (nsteps == 0) return AETH_OK;
  if (c->profile) {
    // timed launches: no graph, events around the dominant kernel
    for (int n = 0; n < nsteps; ++n) {
      aeth_status s = enqueue_step(c, true);
      if (s != AETH_OK) return s;
    }
    return AETH_OK;
  }
  if (!c->graph) {
    // capture one CFL-driven step on a private stream, then replay it
    cudaStream_t cap;
    AETH_CK(c, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaStream_t saved = c->stream;
    c->stream = cap;
    cudaGraph_t g;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    aeth_status s = AETH_OK;
    if (e == cudaSuccess) s = enqueue_step(c, true);
    cudaError_t e2 = cudaStreamEndCapture(cap, &g);
    c->stream = saved;
    cudaStreamDestroy(cap);
    if (e != cudaSuccess || e2 != cudaSuccess)
      return fail(c, AETH_ERR_CUDA, "graph capture failed: %s / %s", cudaGetErrorString(e), cudaGetErrorString(e2));
    if (s != AETH_OK) {
      cudaGraphDestroy(g);
      return s;
    }
    e = cudaGraphInstantiate(&c->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(c, AETH_ERR_CUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
  }
  for (int n = 0; n < nsteps; ++n) AETH_CK(c, cudaGraphLaunch(c->graph, c->stream));
  return AETH_OK;
}

aeth_status aeth_sync(aeth_ctx* c) {
  if (!c) return AETH_ERR_ARG;
  if (!c->finalized) return fail(c, AETH_ERR_STATE, "call aeth_finalize first");
  AETH_CK(c, cudaStreamSynchronize(c->stream));
  AETH_CK(c, cudaGetLastError());
  return read_status(c);
}

aeth_status aeth_diagnostics(aeth_ctx* c, aeth_diag* out) {
  if (!c || !out) return AETH_ERR_ARG;
  if (!c->finalized) return fail(c, AETH_ERR_STATE, "call aeth_finalize first");
  aeth_status s = enqueue_diag(c);
  if (s != AETH_OK) return s;
  double h[6];
  unsigned long long fl = 0, fb = 0;
  AETH_CK(c, cudaMemcpyAsync(h, c->d_diag, sizeof h, cudaMemcpyDeviceToHost, c->stream));
  AETH_CK(c, cudaMemcpyAsync(&fl, c->d_floor, sizeof fl, cudaMemcpyDeviceToHost, c->stream));
  AETH_CK(c, cudaMemcpyAsync(&fb, c->d_fallback, sizeof fb, cudaMemcpyDeviceToHost, c->stream));
  AETH_CK(c, cudaMemsetAsync(c->d_floor, 0, sizeof fl, c->stream));
  AETH_CK(c, cudaMemsetAsync(c->d_fallback, 0, sizeof fb, c->stream));
  AETH_CK(c, cudaStreamSynchronize(c->stream));
  out->mass = h[0];
  out->mom[0] = h[1]; out->mom[1] = h[2]; out->mom[2] = h[3];
  out->energy = h[4];
  out->max_divb_rel = h[5];
  out->floor_hits = (long long)fl;
  out->mlp_fallbacks = (long long)fb;
  return read_status(c);
}

aeth_status aeth_load_mlp(aeth_ctx* c, const float* params, size_t n);

aeth_status aeth_profile(aeth_ctx* c, int enable) {
  if (!c) return AETH_ERR_ARG;
  AETH_CK(c, cudaStreamSynchronize(c->stream));
  c->profile = enable != 0;
  c->prof_used = 0;
  c->prof_bytes = 0;
  c->n_launch = 0;
  return AETH_OK;
}

aeth_status aeth_profile_read(aeth_ctx* c, double* ms, long long* n, double* bytes,
                              long long* all) {
  if (!c) return AETH_ERR_ARG;
  AETH_CK(c, cudaStreamSynchronize(c->stream));
  double tot = 0;
  for (size_t q = 0; q + 1 < c->prof_used; q += 2) {
    float t = 0;
    AETH_CK(c, cudaEventElapsedTime(&t, c->prof_ev[q], c->prof_ev[q + 1]));
    tot += t;
  }
  if (ms) *ms = tot;
  if (n) *n = (long long)(c->prof_used / 2);
  if (bytes) *bytes = c->prof_bytes;
  if (all) *all = c->n_launch;
  return AETH_OK;
}

aeth_status aeth_set_flux_tile(aeth_ctx* c, int flux_tx, int kchunk) {
  if (!c) return AETH_ERR_ARG;
  if (!c->finalized) return fail(c, AETH_ERR_STATE, "call aeth_finalize first");
  if (flux_tx != 32 && flux_tx != 16 && flux_tx != 0)
    return fail(c, AETH_ERR_ARG, "flux tile width 32, 16 or 0 (band tiles)");
  if (!(kchunk >= 1 && kchunk <= 1024)) return fail(c, AETH_ERR_ARG, "z-chunk 1..1024");
  if (flux_tx != 32 && !tile_shape_tunable(c))
    return fail(c, AETH_ERR_UNSUPPORTED, "this configuration keeps the 32-wide flux tile");
  if (flux_tx == 0 && !band_tiles_fit(c))
    return fail(c, AETH_ERR_UNSUPPORTED, "band tiles need blocks at most %d cells wide",
                FLUX_BAND_WMAX - 2);
  c->flux_tx = flux_tx;
  c->kchunk = kchunk;
  aeth_status s = build_tables(c);
  if (s != AETH_OK) return s;
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  return AETH_OK;
}

aeth_status aeth_get_flux_tile(aeth_ctx* c, int* flux_tx, int* kchunk) {
  if (!c) return AETH_ERR_ARG;
  if (!c->finalized) return fail(c, AETH_ERR_STATE, "call aeth_finalize first");
  if (flux_tx) *flux_tx = c->flux_tx;
  if (kchunk) *kchunk = c->kchunk;
  return AETH_OK;
}

aeth_status aeth_autotune(aeth_ctx* c, int* tx_out, int* kchunk_out) {
  if (!c) return AETH_ERR_ARG;
  if (!c->finalized) return fail(c, AETH_ERR_STATE, "call aeth_finalize first");
  // three timed steps per candidate (the state advances, as documented)
  const bool prof = c->profile;
  c->profile = true;
  int best_tx = c->flux_tx, best_kc = c->kchunk;
  double best_ms = 1e300;
  std::vector<int> widths = {32};
  if (tile_shape_tunable(c)) widths.push_back(16);
  if (band_tiles_fit(c)) widths.push_back(0);
  for (int tx : widths) {
    for (int kc : {8, 16, 32, 64}) {
      c->flux_tx = tx;
      c->kchunk = kc;
      aeth_status s = build_tables(c);
      if (s != AETH_OK) return s;
      c->prof_used = 0;
      c->prof_bytes = 0;
      for (int rep = 0; rep < 3; ++rep) {
        s = enqueue_dt(c);
        if (s == AETH_OK) s = enqueue_step(c, false);
        if (s != AETH_OK) return s;
      }
      double ms = 0;
      long long n = 0;
      s = aeth_profile_read(c, &ms, &n, nullptr, nullptr);
      if (s != AETH_OK) return s;
      if (n > 0 && ms / n < best_ms) {
        best_ms = ms / n;
        best_tx = tx;
        best_kc = kc;
      }
    }
  }
  c->flux_tx = best_tx;
  c->kchunk = best_kc;
  aeth_status s = build_tables(c);
  if (s != AETH_OK) return s;
  c->profile = prof;
  c->prof_used = 0;
  c->prof_bytes = 0;
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  if (tx_out) *tx_out = best_tx;
  if (kchunk_out) *kchunk_out = best_kc;
  return AETH_OK;
}

const char* aeth_last_error(const aeth_ctx* c) { return c ? c->err : "null context"; }

void aeth_destroy(aeth_ctx* c) {
  if (!c) return;
  if (c->graph) cudaGraphExecDestroy(c->graph);
  if (c->own_arena && c->arena) cudaFree(c->arena);
  if (c->d_pack) cudaFree(c->d_pack);
  if (c->d_mlp) cudaFree(c->d_mlp);
  if (c->d_mlp_tc) cudaFree(c->d_mlp_tc);
  for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
  delete c;
}

}  // extern "C"
