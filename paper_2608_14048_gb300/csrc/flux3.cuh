// Flux pass of the fused stage (Sec. 2.4): conserved->primitive,
// reconstruction and the Riemann solver for all three face directions of
// every cell in one sweep.  A CTA owns a TX x TY column tile and marches
// along z: each x-y plane of primitives (with the reconstruction halo) is
// staged in a ring of shared-memory planes for the x- and y-faces, while
// every thread keeps the z-stencil of its own column in a register queue
// for the z-faces, filled from the ring.
// Each face is solved exactly once.  Outputs: hydro fluxes, face EMFs (the
// transverse induction fluxes) and the cell-centred reference EMF of the
// upwind CT scheme.
//
// The kernel template lives here so that its instantiations (one per
// Riemann solver family) compile in separate translation units.
#pragma once
#include "runtime.hpp"
#include "stage.cuh"

namespace aeth {

// resident CTAs per SM requested for the FP32 flux pass with donor or PLM
// reconstruction, in 256-thread units (register budget 65536 / (256 *
// FLUX_MINB) per thread: 3, 85 registers, measured 1.3% faster at 256^3
// than 2 with 106 registers); the PPM and PPM5 stencils keep 2 (at 85
// registers they spill about 250 bytes per thread); FP64 takes the whole
// register file.  A 128-thread tile counts half.
#ifndef AETH_FLUX_MINB
#define AETH_FLUX_MINB 3
#endif
// the same for the 128-thread 2-D tiles, in CTAs: 5 (the PLM corrector at
// 96 registers with a 20-byte spill) measured 1% faster at 256^3 than 6
// (80 registers, 160 bytes spilled); PPM keeps 4
#ifndef AETH_FLUX_MINB_2D
#define AETH_FLUX_MINB_2D 5
#endif
#ifndef AETH_FLUX_MINB_2D_PPM
#define AETH_FLUX_MINB_2D_PPM 4
#endif
template <typename R, int RECON>
__host__ __device__ constexpr int flux_minb(int txt) {
  return txt == 0 ? (sizeof(R) == 4 ? (RECON >= 2 ? 2 : AETH_FLUX_MINB) : 1)
                  : (sizeof(R) == 4 ? (RECON >= 2 ? AETH_FLUX_MINB_2D_PPM : AETH_FLUX_MINB_2D) : 2);
}

__host__ __device__ __forceinline__ int ceil_div_d(int a, int b) { return (a + b - 1) / b; }

// Shared-memory plane (one variable, tile + halo) of a band tile (TXT = 0,
// see band_rows): the largest (rows + halo) x (width + halo) over the
// widths a band tile takes, so that its stride is a compile-time constant.
__host__ __device__ constexpr int band_smem(int halo) {
  int m = 0;
  for (int w = 3; w <= FLUX_BAND_WMAX; ++w) {
    const int a = (band_rows(w - 2) + halo) * (w + halo);
    m = a > m ? a : m;
  }
  return m;
}

// Values of one staged variable plane of a flux tile TXT wide (0: band).
template <int RECON>
__host__ __device__ constexpr int flux_plane(int txt) {
  return txt ? (txt + 2 * recon_reach<RECON>() + 1) * (FLUX_NT / txt + 2 * recon_reach<RECON>() + 1)
             : band_smem(2 * recon_reach<RECON>() + 1);
}

// Planes in the shared-memory ring of a 2-D flux tile: the z-queue takes
// plane k + RH while the x- and y-faces read plane k, and the next plane is
// staged while slower warps still read plane k - 1.  Band tiles stage one
// plane at a time (two barriers per plane, the z queue from memory): on the
// small blocks they serve, the ring's larger shared-memory footprint cost
// more in L1 hits than its one barrier per plane saved.
template <int RECON>
__host__ __device__ constexpr int flux_ring(int txt) { return txt ? recon_reach<RECON>() + 2 : 1; }

// Solver families 3 and 4 are the isothermal ones.
constexpr bool iso_solver(int solver) { return solver == 3 || solver == 4; }

// Riemann solver family SOLVER (numbering of k_flux3 below) on one face.
template <int SOLVER, typename R>
__device__ __forceinline__ void solve_face(R g, const R* wl, const R* wr, R bn, R* fx) {
  if constexpr (SOLVER == 2) hlle(g, wl, wr, bn, fx);
  else if constexpr (SOLVER == 3) hlld_iso(g, wl, wr, bn, fx);
  else if constexpr (SOLVER == 4) hlle_iso(g, wl, wr, bn, fx);
  else if constexpr (SOLVER == 5) hlld<true>(g, wl, wr, bn, fx);
  else hlld(g, wl, wr, bn, fx);
}

// Store the outputs of one face of direction D.  Scratch arrays sit at
// sb + slot * pitch: E_ref 0..2, fluxes 8 + 5 D + v, face EMFs 23 + 2 D + q.
template <int D, typename R>
__device__ __forceinline__ void store_face(R* __restrict__ sb, long long pitch, long long fc,
                                           const R* fx) {
  constexpr int T1 = (D + 1) % 3, T2 = (D + 2) % 3;
  R* f = sb + (8 + 5 * D) * pitch + fc;
  f[0] = fx[0];
  f[(1 + D) * pitch] = fx[1];
  f[(1 + T1) * pitch] = fx[2];
  f[(1 + T2) * pitch] = fx[3];
  f[4 * pitch] = fx[4];
  R* e = sb + (23 + 2 * D) * pitch + fc;
  e[0] = fx[6];        // E_t1 =  F(B_t2)
  e[pitch] = -fx[5];   // E_t2 = -F(B_t1)
}

// ------------------------------------------------------------------------
// 1. flux pass.  Persistent: CTAs stride over the tiles of all blocks.
//    AETH_FLUX_MINB CTAs per SM in FP32; FP64 takes the full register file.
// ------------------------------------------------------------------------
// SOLVER 0: HLLD; 2: HLLE; 1: write the face states (wl, wr, bn) for the
// learned flux instead of solving; 3: isothermal HLLD; 4: isothermal HLLE;
// 5: the low-dissipation HLLD (LHLLD).  For the isothermal solvers the
// `gamma` argument carries the sound speed cs, the primitive pressure is
// cs^2 rho and is not reconstructed (the isothermal fluxes take the
// pressure from the reconstructed density).
// DUAL: dual energy (Sec. 2.8): the pressure of an untrusted internal energy
// (below alpha_switch x kinetic + magnetic) comes from the entropy, and each
// face also gets the entropy flux, its mass flux times the reconstructed
// specific entropy S/rho of the upwind side, in scratch slot 3 + D.
// TXT: the tile's x width (32 or 16; y width NT / TXT), or 0 for a band
// tile: whole rows of the block (x from -1 to n_x), band_rows(n_x) of them,
// so that a block narrower than the 2-D tile keeps its lanes busy.
// Dynamic shared memory: flux_ring<RECON>(TXT) x NW planes of
// flux_plane<RECON>(TXT) values.
template <typename R, bool P64, int RECON, bool MHD, typename Src, int SOLVER = 0,
          bool DUAL = false, int TXT = FLUX_TX>
__global__ void __launch_bounds__(flux_threads(TXT), (flux_minb<R, RECON>(TXT)))
    k_flux3(Src S, int t0, int t1, int src, R gamma, R rho_floor, R p_floor, int kchunk,
            unsigned long long* floor_hits, R alpha_switch) {
  constexpr bool BAND = TXT == 0;
  constexpr int NT = flux_threads(TXT);
  constexpr int TX = BAND ? 1 : TXT, TY = NT / TX;
  constexpr int RH = recon_reach<RECON>(), RL = RH + 1;
  constexpr int WX = TX + RL + RH, WY = TY + RL + RH;
  constexpr int QN = RL + RH + 1;
  constexpr int NB = flux_ring<RECON>(TXT);
  constexpr bool RING = NB > 1;
  constexpr int NW = NPRIM + (DUAL ? 1 : 0);   // staged variables (+ S/rho)
  constexpr int NQ = 7 + (DUAL ? 1 : 0);       // z-queue variables (+ S/rho)
  extern __shared__ __align__(16) unsigned char flux_smem[];
  R* __restrict__ sw = reinterpret_cast<R*>(flux_smem);
  constexpr int SN = flux_plane<RECON>(TXT);   // values of one staged plane
  // variable v of ring plane b at plane offset s (row pitch wxr)
  auto at = [&](int b, int v, int s) -> R& { return sw[(b * NW + v) * SN + s]; };
  constexpr bool ISO = iso_solver(SOLVER);
  const R gm1 = ISO ? gamma * gamma : gamma - R(1);   // cs^2 for ISO
  int hits = 0;

  for (int t = t0 + (int)blockIdx.x; t < t1; t += gridDim.x) {
    int loc;
    const BlockPtrs<R>& P = S.get(t, loc);
    const Layout L = P.L;
    const R* __restrict__ ub = P.reg[src][0];   // state arrays at ub + v * pitch
    const R* __restrict__ eb = P.ent[src];       // entropy (DUAL)
    R* __restrict__ sb = P.w[0];                 // scratch arrays at sb + slot * pitch
    const long long pitch = P.pitch;
    const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
    int i0, j0, bz, tx, ty, wxr, wyr;
    if constexpr (BAND) {
      const int W = nx + 2, br = band_rows(nx);
      const int nb = ceil_div_d(ny + 2, br);
      bz = loc / nb;
      i0 = -1;
      j0 = -1 + (loc % nb) * br;
      tx = (int)threadIdx.x % W;
      ty = (int)threadIdx.x / W;   // >= br: an idle thread of the band
      wxr = W + RL + RH;
      wyr = br + RL + RH;
    } else {
      const int ntx = ceil_div_d(nx + 2, TX), nty = ceil_div_d(ny + 2, TY);
      const int bx = loc % ntx, by = (loc / ntx) % nty;
      bz = loc / (ntx * nty);
      i0 = -1 + bx * TX;
      j0 = -1 + by * TY;
      tx = (int)threadIdx.x % TX;
      ty = (int)threadIdx.x / TX;
      wxr = WX;
      wyr = WY;
    }
    const int i = i0 + tx, j = j0 + ty;
    const int k0 = -1 + bz * kchunk;
    const int k1 = min(nz, k0 + kchunk - 1);
    const bool active =
        i <= nx && j <= ny && (!BAND || ty < band_rows(nx));

    // primitives of cell cc (+ specific entropy sp with DUAL); returns floor hits
    auto prim_at = [&](long long cc, R* w, R& sp) -> int {
      if constexpr (DUAL) {
        return prim_cell_dual<R, MHD>(L, ub, pitch, eb, cc, gm1, rho_floor, p_floor, alpha_switch,
                                      w, sp);
      } else {
        sp = R(0);
        return prim_cell_s<R, P64, MHD, ISO>(L, ub, pitch, cc, gm1, rho_floor, p_floor, w);
      }
    };
    // z register queue of the own column: planes k-RL .. k+RH, 7 variables
    // (+ S/rho; the z-face normal field comes from the face array), in the
    // z-face frame order rho, vz, vx, vy, p, Bx, By
    R q[NQ][QN];
    auto load_q = [&](int slot, int kk) {   // from memory (planes below the chunk)
      R w[8], sp = R(1);
      if (active && in_prim_range(L, i, j, kk)) {
        prim_at(L.idx(i, j, kk), w, sp);
      } else {
        w[0] = R(1); w[1] = w[2] = w[3] = R(0); w[4] = R(1); w[5] = w[6] = w[7] = R(0);
      }
      q[0][slot] = w[0]; q[1][slot] = w[3]; q[2][slot] = w[1]; q[3][slot] = w[2];
      q[4][slot] = w[4]; q[5][slot] = w[5]; q[6][slot] = w[6];
      if constexpr (DUAL) q[NQ - 1][slot] = sp;
    };
    const int sx = tx + RL, sy = ty + RL, so = sy * wxr + sx;   // own cell in a plane
    auto ring_q = [&](int slot, int b) {    // from the staged plane in ring slot b
      if (!active) return;
      q[0][slot] = at(b, 0, so); q[1][slot] = at(b, 3, so); q[2][slot] = at(b, 1, so);
      q[3][slot] = at(b, 2, so); q[4][slot] = at(b, 4, so); q[5][slot] = at(b, 5, so);
      q[6][slot] = at(b, 6, so);
      if constexpr (DUAL) q[NQ - 1][slot] = at(b, NW - 1, so);
    };
    // stage plane kk (tile + halo) into ring slot b
    auto stage = [&](int kk, int b) {
      for (int s = threadIdx.x; s < wxr * wyr; s += NT) {
        const int rx = s % wxr, ry = s / wxr;
        const int ci = i0 - RL + rx, cj = j0 - RL + ry;
        R w[8], sp = R(1);
        if (in_prim_range(L, ci, cj, kk)) {
          const int h = prim_at(L.idx(ci, cj, kk), w, sp);
          if (kk <= k1) hits += h;   // the planes above the chunk are the next one's
        } else {
          w[0] = R(1); w[1] = w[2] = w[3] = R(0); w[4] = R(1); w[5] = w[6] = w[7] = R(0);
        }
#pragma unroll
        for (int v = 0; v < NPRIM; ++v) at(b, v, s) = w[v];
        if constexpr (DUAL) at(b, NW - 1, s) = sp;
      }
    };
    // the previous tile's last plane is read until every warp is past here
    __syncthreads();
    if constexpr (RING) {
#pragma unroll
      for (int s = 0; s < RL; ++s) load_q(s, k0 - RL + s);
#pragma unroll
      for (int m = 0; m < RH; ++m) stage(k0 + m, m);
    } else {
#pragma unroll
      for (int s = 0; s < QN - 1; ++s) load_q(s + 1, k0 - RL + s);
    }
    for (int k = k0; k <= k1; ++k) {
      int bk = 0;
      if constexpr (RING) {
        // plane k + RH goes to ring slot (k - k0 + RH) % NB, which last held
        // plane k - 2, read by no warp past the previous barrier: one
        // barrier per plane, and each warp stages the next plane as soon as
        // its faces are done
        const int m = k - k0;
        const int bq = (m + RH) % NB;
        bk = m % NB;
        stage(k + RH, bq);
        __syncthreads();
        if (m == 0) {
#pragma unroll
          for (int s = 0; s <= RH; ++s) ring_q(RL + s, s);
        } else {
          // advance the z queue: drop plane k-RL-1, add plane k+RH
#pragma unroll
          for (int v = 0; v < NQ; ++v)
#pragma unroll
            for (int s = 0; s < QN - 1; ++s) q[v][s] = q[v][s + 1];
          ring_q(QN - 1, bq);
        }
      } else {
        // one staged plane, the z queue from memory
        if (k > k0) __syncthreads();
        stage(k, 0);
#pragma unroll
        for (int v = 0; v < NQ; ++v)
#pragma unroll
          for (int s = 0; s < QN - 1; ++s) q[v][s] = q[v][s + 1];
        load_q(QN - 1, k + RH);
        __syncthreads();
      }
      if (!active) continue;

      // the faces of plane k from ring slot bk (x, y, E_ref) and the z queue
      const long long fc = L.idx(i, j, k);
      R wl[7], wr[7], fx[7];
      // ---- x-face (i-1/2, j, k): frame (rho, vx, vy, vz, p, By, Bz)
      if (i >= 0) {
        const int slot[7] = {0, 1, 2, 3, 4, 6, 7};
#pragma unroll
        for (int v = 0; v < 7; ++v) {
          if ((!MHD && v >= 5) || (ISO && v == 4)) { wl[v] = wr[v] = R(0); continue; }
          recon_var<RECON>([&](int off) { return at(bk, slot[v], so + off); }, wl[v], wr[v]);
        }
        const R bn = MHD ? ub[5 * pitch + fc] : R(0);
        if (SOLVER != 1) {
          solve_face<SOLVER>(gamma, wl, wr, bn, fx);
          store_face<0>(sb, pitch, fc, fx);
          if constexpr (DUAL) {
            R sl, sr;
            recon_var<RECON>([&](int off) { return at(bk, NW - 1, so + off); }, sl, sr);
            sb[3 * pitch + fc] = fx[0] >= R(0) ? fx[0] * sl : fx[0] * sr;
          }
        } else {
          R* fs = P.fstate + (0 * 15) * pitch + fc;
#pragma unroll
          for (int v = 0; v < 7; ++v) { fs[v * pitch] = wl[v]; fs[(7 + v) * pitch] = wr[v]; }
          fs[14 * pitch] = bn;
        }
      }
      // ---- y-face (i, j-1/2, k): frame (rho, vy, vz, vx, p, Bz, Bx)
      if (j >= 0) {
        const int slot[7] = {0, 2, 3, 1, 4, 7, 5};
#pragma unroll
        for (int v = 0; v < 7; ++v) {
          if ((!MHD && v >= 5) || (ISO && v == 4)) { wl[v] = wr[v] = R(0); continue; }
          recon_var<RECON>([&](int off) { return at(bk, slot[v], so + off * wxr); }, wl[v], wr[v]);
        }
        const R bn = MHD ? ub[6 * pitch + fc] : R(0);
        if (SOLVER != 1) {
          solve_face<SOLVER>(gamma, wl, wr, bn, fx);
          store_face<1>(sb, pitch, fc, fx);
          if constexpr (DUAL) {
            R sl, sr;
            recon_var<RECON>([&](int off) { return at(bk, NW - 1, so + off * wxr); }, sl, sr);
            sb[4 * pitch + fc] = fx[0] >= R(0) ? fx[0] * sl : fx[0] * sr;
          }
        } else {
          R* fs = P.fstate + (1 * 15) * pitch + fc;
#pragma unroll
          for (int v = 0; v < 7; ++v) { fs[v * pitch] = wl[v]; fs[(7 + v) * pitch] = wr[v]; }
          fs[14 * pitch] = bn;
        }
      }
      // ---- z-face (i, j, k-1/2): frame (rho, vz, vx, vy, p, Bx, By)
      if (k >= 0) {
#pragma unroll
        for (int v = 0; v < 7; ++v) {
          if ((!MHD && v >= 5) || (ISO && v == 4)) { wl[v] = wr[v] = R(0); continue; }
          recon_var<RECON>([&](int off) { return q[v][off + RL]; }, wl[v], wr[v]);
        }
        const R bn = MHD ? ub[7 * pitch + fc] : R(0);
        if (SOLVER != 1) {
          solve_face<SOLVER>(gamma, wl, wr, bn, fx);
          store_face<2>(sb, pitch, fc, fx);
          if constexpr (DUAL) {
            R sl, sr;
            recon_var<RECON>([&](int off) { return q[NQ - 1][off + RL]; }, sl, sr);
            sb[5 * pitch + fc] = fx[0] >= R(0) ? fx[0] * sl : fx[0] * sr;
          }
        } else {
          R* fs = P.fstate + (2 * 15) * pitch + fc;
#pragma unroll
          for (int v = 0; v < 7; ++v) { fs[v * pitch] = wl[v]; fs[(7 + v) * pitch] = wr[v]; }
          fs[14 * pitch] = bn;
        }
      }
      // ---- cell-centred reference EMF, E = -v x B
      if (MHD) {
        const R vx = at(bk, 1, so), vy = at(bk, 2, so), vz = at(bk, 3, so);
        const R bx_ = at(bk, 5, so), by_ = at(bk, 6, so), bz_ = at(bk, 7, so);
        sb[fc] = -(vy * bz_ - vz * by_);
        sb[pitch + fc] = -(vz * bx_ - vx * bz_);
        sb[2 * pitch + fc] = -(vx * by_ - vy * bx_);
      }
    }
  }
  if (hits) atomicAdd(floor_hits, (unsigned long long)hits);
}

// ------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------
struct TileRange {
  int t0, t1;
};

static TileRange range_of(const aeth_ctx* c, int kind, int block) {
  const int nb = (int)c->blocks.size();
  const int* p = c->h_prefix.data() + kind * (nb + 1);
  if (block < 0) return {0, p[nb]};
  return {p[block], p[block + 1]};
}

template <typename R>
static const BlockPtrs<R>* dtab(const aeth_ctx* c) {
  return (const BlockPtrs<R>*)c->d_tab;
}

static const int* dpre(const aeth_ctx* c, int kind) {
  return c->d_prefix + kind * ((int)c->blocks.size() + 1);
}

// Launch a pass either from the device table (several blocks) or with the
// block's pointers in the kernel parameters (one block).
template <typename R, typename F>
static void with_src(aeth_ctx* c, int kind, int block, F launch) {
  const int nb = (int)c->blocks.size();
  if (nb == 1 || block >= 0) {
    const int b = block >= 0 ? block : 0;
    const TileRange r = range_of(c, kind, b);
    launch(ParamSrc<R>{block_ptrs<R>(c, b), r.t0}, r);
  } else {
    launch(TableSrc<R>{dtab<R>(c), dpre(c, kind), nb, c->d_tmap[kind]}, range_of(c, kind, -1));
  }
}

template <typename R, bool P64, int RECON, bool MHD, int SOLVER, bool DUAL>
static void launch_flux3(aeth_ctx* c, int src, int block) {

  constexpr int NW = NPRIM + (DUAL ? 1 : 0);
  with_src<R>(c, PK_FLUX, block, [&](auto S, TileRange r) {
    // tx: the tile width the kernel was built for (0: band tiles)
    auto go = [&](auto kernel, int tx) {
      const int per_sm = flux_minb<R, RECON>(tx);
      const int grid = std::max(1, std::min(r.t1 - r.t0, c->num_sms * per_sm));
      const int bytes = flux_ring<RECON>(tx) * NW * flux_plane<RECON>(tx) * (int)sizeof(R);
      // above the 48 KB default (FP64, PPM rings, bands); a plain attribute
      // call, also legal while a graph is being captured
      if (bytes > 48 * 1024)
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
      kernel<<<grid, flux_threads(tx), bytes, c->stream>>>(
          S, r.t0, r.t1, src, (R)(iso_solver(SOLVER) ? c->cfg.cs_iso : c->cfg.gamma),
          (R)c->cfg.rho_floor, (R)c->cfg.p_floor, c->kchunk, c->d_floor,
          (R)c->cfg.alpha_switch);
    };
    // the 16-wide tile is built for the FP32 solver passes (the contexts
    // whose tiles the autotuner may switch: tile_shape_tunable)
    if constexpr (sizeof(R) == 4 && !DUAL && SOLVER != 1) {
      if (c->flux_tx == 16) {
        go(k_flux3<R, P64, RECON, MHD, decltype(S), SOLVER, DUAL, 16>, 16);
        return;
      }
      if (c->flux_tx == 0) {
        go(k_flux3<R, P64, RECON, MHD, decltype(S), SOLVER, DUAL, 0>, 0);
        return;
      }
    }
    go(k_flux3<R, P64, RECON, MHD, decltype(S), SOLVER, DUAL, 32>, 32);
  });
  c->n_launch += 1;
}

// One flux pass with the solver family SOLVER and the reconstruction of the
// context (explicitly instantiated per family in flux_*.cu; DUAL in
// flux_dual_*.cu).
template <typename R, bool P64, bool MHD, int SOLVER, bool DUAL = false>
void flux_pass_solver(aeth_ctx* c, int recon, int src, int block);

template <typename R, bool P64, bool MHD, int SOLVER, bool DUAL>
void flux_pass_solver_impl(aeth_ctx* c, int recon, int src, int block) {
  if (recon == AETH_RECON_DONOR) launch_flux3<R, P64, 0, MHD, SOLVER, DUAL>(c, src, block);
  else if (recon == AETH_RECON_PLM) launch_flux3<R, P64, 1, MHD, SOLVER, DUAL>(c, src, block);
  else if (recon == AETH_RECON_PPM5) launch_flux3<R, P64, 3, MHD, SOLVER, DUAL>(c, src, block);
  else launch_flux3<R, P64, 2, MHD, SOLVER, DUAL>(c, src, block);
}

}  // namespace aeth
