/*
 * aether_gb.h -- C ABI of the GB300 (sm_103a) finite-volume MHD step.
 *
 * The library advances the ideal-MHD equations (paper Sec. 2.1, Eqs. 1-5) on
 * one GPU with the unsplit Godunov scheme of the Aether.jl paper
 * (arXiv 2608.14048): per-direction reconstruction of primitive variables
 * and HLLD Riemann fluxes (Sec. 2.4), the finite-volume update of Eq. 8,
 * constrained transport of face-centred B with upwinded corner EMFs (Sec. 2.5,
 * Eq. 9), a two-stage predictor-corrector (Sec. 2.6), and the CFL step of
 * Eq. 11.  Multifluid dust (Sec. 2.2) advances with IMEX2P and a closed-form
 * implicit drag solve.
 *
 * Conventions shared by every call
 * --------------------------------
 * - Return value: AETH_OK (0) or a negative aeth_status.  aeth_last_error()
 *   gives a human-readable reason for the last failure on that context.
 * - Host arrays passed in or out are caller-owned FP64, row-major with i
 *   fastest: cons[5][nz][ny][nx] = (rho, M1, M2, M3, E);
 *   b1[nz][ny][nx+1], b2[nz][ny+1][nx], b3[nz+1][ny][nx] are the face-averaged
 *   normal field components.  Along a periodic axis the last face is the
 *   image of the first (the library reads the first, writes both).
 *   The library converts to its working precision on the device.  Pinned
 *   host memory makes the copies asynchronous-fast; pageable memory works.
 * - Device memory belongs to the library (cudaMalloc at aeth_finalize) or to
 *   a caller-provided arena (aeth_bind_arena), which must outlive the ctx.
 * - All device work is enqueued on the bound CUDA stream (default: the
 *   legacy default stream).  aeth_step is asynchronous; device-side errors
 *   (non-finite state, floors hit in strict mode) are latched in a device
 *   status word and returned by the next aeth_sync, aeth_compute_dt,
 *   aeth_get_state or aeth_diagnostics.
 * - A context is not thread-safe; distinct contexts are independent.
 */
#ifndef AETHER_GB_H
#define AETHER_GB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct aeth_ctx aeth_ctx; /* opaque; owned by the library */

typedef enum {
  AETH_OK = 0,
  AETH_ERR_ARG = -1,         /* invalid argument or size */
  AETH_ERR_OOM = -2,         /* device or host allocation failed */
  AETH_ERR_CUDA = -3,        /* a CUDA runtime call failed */
  AETH_ERR_NONFINITE = -4,   /* NaN/Inf found in the state */
  AETH_ERR_FLOOR = -5,       /* floors applied while strict_floors = 1 */
  AETH_ERR_TIMEOUT = -6,     /* a bounded device wait gave up */
  AETH_ERR_STATE = -7,       /* call out of order (e.g. step before finalize) */
  AETH_ERR_UNSUPPORTED = -8  /* option combination not built */
} aeth_status;

/* equation of state (Sec. 2.1): ideal gas p = (gamma - 1) e, or the
 * isothermal closure p = cs_iso^2 rho (no energy equation: the energy slot
 * of the state is carried with zero flux; the isothermal HLLD of Mignone
 * (2007) or the isothermal HLLE solves the faces; gas only) */
enum {
  AETH_EOS_ADIABATIC_MHD = 0,
  AETH_EOS_ADIABATIC_HYDRO = 1,
  AETH_EOS_ISOTHERMAL_MHD = 2,
  AETH_EOS_ISOTHERMAL_HYDRO = 3
};
/* reconstruction (Sec. 2.4): donor cell, PLM (van Leer 1974 limiter), PPM
 * (Colella & Woodward 1984), PPM5 (interface values from the quartic
 * through the five cell averages centred on each cell, with the PPM
 * limiter; 3 ghost layers like PPM) */
enum { AETH_RECON_DONOR = 0, AETH_RECON_PLM = 1, AETH_RECON_PPM = 2, AETH_RECON_PPM5 = 3 };
/* Riemann solver (Sec. 2.4): HLLD (Miyoshi & Kusano 2005); HLLE (Harten,
 * Lax & van Leer 1983; Einfeldt 1988) with the outer speed estimates of the
 * HLLD solver, the paper's throughput-benchmark solver; AETH_RIEMANN_MLP =
 * learned flux with HLLD fallback; AETH_RIEMANN_LHLLD = low-dissipation HLLD
 * (after Minoshima & Miyoshi 2021): HLLD with the pressure dissipation at the
 * contact (normal-momentum and energy flux) scaled by the local Mach number
 * phi = min(1, max|v| / max c_f); LHLLC in hydro mode; adiabatic closures */
enum { AETH_RIEMANN_HLLD = 0, AETH_RIEMANN_HLLE = 1, AETH_RIEMANN_MLP = 2,
       AETH_RIEMANN_LHLLD = 3 };
/* tensor-core engine of the learned flux: tcgen05 MMAs with TMEM
 * accumulators, or warp-level mma.sync */
enum { AETH_MLP_TCGEN05 = 0, AETH_MLP_MMA_SYNC = 1 };
/* time integrator (Sec. 2.6): VL2, SSP-RK2, IMEX2P (dust runs), SSP-RK3
 * (three stages in the two registers; Cartesian blocks only, since its
 * middle stage updates the stage register in place) */
enum { AETH_INT_VL2 = 0, AETH_INT_RK2 = 1, AETH_INT_IMEX2P = 2, AETH_INT_RK3 = 3 };
/* working precision: all-FP64; FP32; FP32 with the pressure recovery of
 * Eq. 5 (E minus kinetic minus magnetic energy) evaluated in FP64 in every
 * cell; FP32 with that FP64 recovery only in the cells that need it
 * (AETH_FP32_SEL64: where kinetic + magnetic energy exceeds p64_ratio
 * times the internal energy, so that the FP32 subtraction would lose more
 * than a few bits -- low plasma beta or high Mach number; every other cell
 * takes the FP32 recovery) */
enum { AETH_FP64 = 0, AETH_FP32 = 1, AETH_FP32_P64 = 2, AETH_FP32_SEL64 = 3 };
/* precision of the implicit drag solve of dust runs (drag_precision) */
enum { AETH_DRAG_FP64 = 0, AETH_DRAG_FP32 = 1, AETH_DRAG_SEL64 = 2 };
/* drag law of dust runs (Sec. 2.2): constant stopping times t_k, or constant
 * drag coefficients K_k with t_k = rho_k / K_k (the law of the paper's
 * steady dusty shock, Sec. 5.8.2) */
enum { AETH_DRAG_LAW_TSTOP = 0, AETH_DRAG_LAW_COEFF = 1 };
/* coordinates (Sec. 2.3) */
enum { AETH_COORD_CART = 0, AETH_COORD_SPH = 1 };
/* boundary kind per axis, both sides (Sec. 2.3) */
enum { AETH_BC_PERIODIC = 0, AETH_BC_OUTFLOW = 1 };
/* kernel path */
enum { AETH_PATH_FUSED = 0, AETH_PATH_UNFUSED = 1 };

typedef struct {
  int eos;            /* AETH_EOS_* */
  double gamma;       /* adiabatic index of the ideal-gas closure (> 1; not
                         read by the isothermal closure) */
  double rho_floor;   /* density floor of the cons->prim conversion */
  double p_floor;     /* pressure floor */
  int recon;          /* AETH_RECON_* of the final stage */
  int riemann;        /* AETH_RIEMANN_* */
  int integrator;     /* AETH_INT_* */
  double cfl;         /* Courant factor C of Eq. 11 */
  int precision;      /* AETH_FP64 / AETH_FP32 / AETH_FP32_P64 / AETH_FP32_SEL64 */
  int path;           /* AETH_PATH_FUSED (default) or AETH_PATH_UNFUSED */
  int strict_floors;  /* 1: a floor hit latches AETH_ERR_FLOOR */
  int n_dust;         /* number of pressureless dust species (0: none); the
                         gas is adiabatic or isothermal hydro, IMEX2P */
  const double* t_stop; /* [n_dust] constant stopping times t_k, or with
                           drag_law = AETH_DRAG_LAW_COEFF the drag
                           coefficients K_k (copied; each > 0) */
  int drag_precision; /* AETH_DRAG_FP64 (default, 0): implicit drag solve in
                         FP64; AETH_DRAG_FP32: in FP32; AETH_DRAG_SEL64: in
                         FP64 only for the species whose implicit weight
                         h / t_k (h = the stage's implicit step) exceeds
                         drag_ratio, in FP32 for the others (dust runs
                         only; AETH_FP64 and AETH_FP32 keep their values) */
  double mlp_tau;     /* learned flux: residual-check tolerance (fraction of the
                         HLL dissipation bracket); <= 0 selects 0.25 */
  int mlp_engine;     /* learned flux: AETH_MLP_TCGEN05 (default, 0) or
                         AETH_MLP_MMA_SYNC */
  double cs_iso;      /* isothermal sound speed (> 0, finite) of the
                         AETH_EOS_ISOTHERMAL_* closures; ignored otherwise */
  int dual_energy;    /* 1: dual-energy formalism (Sec. 2.8, Bryan 1995 in the
                         entropy form): the entropy S = p / rho^(gamma-1) is
                         advected alongside the state (mass flux x S/rho of
                         the upwind side); at every stage start a cell whose
                         internal energy E - kinetic - magnetic is below
                         alpha_switch x (kinetic + magnetic) takes its
                         pressure from S and has E rewritten to match, one
                         above alpha_sync x (kinetic + magnetic) has S
                         resynchronised from E.  Adiabatic closures, fused
                         path, AETH_FP64 or AETH_FP32 (it is the alternative
                         to AETH_FP32_P64), HLLD / HLLE / LHLLD, no dust.
                         S is initialised from the state by aeth_set_state
                         and read back with aeth_get_entropy. */
  double alpha_switch; /* <= 0 selects 1e-3 */
  double alpha_sync;   /* <= 0 selects 1e-1 */
  double p64_ratio;    /* AETH_FP32_SEL64: a cell takes the FP64 pressure
                          recovery where (kinetic + magnetic) > p64_ratio x
                          internal energy (its FP32 estimate); <= 0 selects
                          4, where the FP32 subtraction's relative error,
                          about 4 ulp x the ratio, stays below 1e-6 */
  double drag_ratio;   /* AETH_DRAG_SEL64: species with h / t_k > drag_ratio
                          are solved in FP64; <= 0 selects 1 */
  int drag_law;        /* AETH_DRAG_LAW_TSTOP (default, 0) or
                          AETH_DRAG_LAW_COEFF; the latter takes a_k =
                          h K_k / rho_k per cell (a species with rho_k <= 0
                          feels no drag) and not AETH_DRAG_SEL64 */
} aeth_config;

typedef struct {
  int nx, ny, nz;     /* interior cells along x1, x2, x3 (each >= 1) */
  int coord;          /* AETH_COORD_* */
  double x1min, x1max, x2min, x2max, x3min, x3max;
  int bc[3];          /* AETH_BC_* per axis */
} aeth_block_desc;

typedef struct {
  double mass;          /* sum rho V over all blocks */
  double mom[3];        /* sum M_d V */
  double energy;        /* sum E V */
  double max_divb_rel;  /* max over cells |sum_f +-A_f B_f| / sum_f A_f|B_f| */
  long long floor_hits; /* cells floored since the last diagnostics call */
  long long mlp_fallbacks; /* faces recomputed with HLLD by the MLP path */
} aeth_diag;

/* Create a context from a configuration (Sec. 3.4 "Simulation(...)").
 * Copies everything it needs from *cfg.  Errors: AETH_ERR_ARG for invalid
 * enums/values, AETH_ERR_UNSUPPORTED for combinations not built. */
aeth_status aeth_create(const aeth_config* cfg, aeth_ctx** out);

/* Execution backend (Sec. 3.4: the Mesh constructor names the backend a run
 * executes on; Sec. 3.2: every kernel is launched on it).  Here the backend
 * is one CUDA stream: enqueue all further device work on `cuda_stream` (a
 * cudaStream_t, e.g. torch.cuda.current_stream().cuda_stream); NULL = legacy
 * default stream.  AETH_ERR_ARG for a NULL ctx. */
aeth_status aeth_bind_stream(aeth_ctx* ctx, void* cuda_stream);

/* Device memory of the state (Sec. 3.3: on GPU systems the solver's arrays,
 * ghost zones included, live in device memory).  Use [dev_ptr, dev_ptr +
 * bytes) as the device arena instead of allocating.  Must be called before
 * aeth_finalize; dev_ptr must be 256-byte aligned and outlive the context;
 * the caller keeps ownership.  Query the size with aeth_plan.
 * AETH_ERR_STATE after aeth_finalize, AETH_ERR_ARG for a misaligned
 * pointer. */
aeth_status aeth_bind_arena(aeth_ctx* ctx, void* dev_ptr, size_t bytes);

/* Add one mesh block (Sec. 2.3; blocks may differ in size, coordinates and
 * boundary kinds).  Blocks are independent boxes: ghost zones are filled
 * from each block's own boundary conditions.  Returns its id (0, 1, ...)
 * in *block_id. */
aeth_status aeth_add_block(aeth_ctx* ctx, const aeth_block_desc* desc,
                           int* block_id);

/* Mesh-block decomposition (Sec. 2.3): block `hi` lies beyond the upper
 * face of block `lo` along `axis` (0, 1, 2), so the two share that face.
 * Each block's ghost cells (and ghost faces) on a linked side are copied
 * from the neighbour's cells, in one fill pass over all blocks per axis,
 * which also supplies the edge and corner ghosts; the shared face's normal
 * field is updated by the block above and mirrored into face n of the block
 * below.  A linked side ignores the block's bc on that side; a block
 * linked to itself is periodic along that axis.  Both blocks Cartesian,
 * with equal cell counts across the face and >= ghost-width cells along
 * `axis`; fused path, gas only.  Call after aeth_add_block, before
 * aeth_plan.  AETH_ERR_ARG for bad indices, an already linked side or
 * mismatched blocks; AETH_ERR_UNSUPPORTED for spherical blocks, the unfused
 * path or dust. */
aeth_status aeth_link_blocks(aeth_ctx* ctx, int lo, int axis, int hi);

/* Close the mesh description (Sec. 3.4: the Mesh constructor fixes the
 * domain, resolution and block decomposition before any state exists) and
 * compute the device-memory layout; *bytes_needed receives the arena size.
 * Host only: no CUDA call.  AETH_ERR_STATE when no block was added. */
aeth_status aeth_plan(aeth_ctx* ctx, size_t* bytes_needed);

/* Complete the Mesh/Simulation construction of Sec. 3.4: lay out device
 * memory (in the bound arena, else cudaMalloc) and build the launch tables
 * of every block (Sec. 2.3).  *bytes_needed (may be NULL) receives the
 * size.  AETH_ERR_ARG if a bound arena is too small, AETH_ERR_OOM if the
 * allocation fails. */
aeth_status aeth_finalize(aeth_ctx* ctx, size_t* bytes_needed);

/* Initial condition of one block (Sec. 3.4, the set_initial_condition!
 * step of the problem setup): copy the conserved variables of Eq. 1 and the
 * face-averaged field of Eq. 9 from host FP64 arrays (layout above) to the
 * device, converting to the working precision.  The face field should come
 * from a vector potential (Sec. 3.4) so that div B starts at round-off.
 * Synchronous with respect to the host arrays (they may be reused when the
 * call returns).  AETH_ERR_STATE before aeth_finalize, AETH_ERR_ARG for a
 * bad block index or NULL cons (b1f..b3f may be NULL in hydro). */
aeth_status aeth_set_state(aeth_ctx* ctx, int block, const double* cons,
                           const double* b1f, const double* b2f,
                           const double* b3f);

/* Read the state back (Sec. 3.4: the state stays inspectable after run!
 * returns): copy one block's conserved variables and face field to host
 * FP64 arrays (layout above; caller-owned).  Synchronises the stream;
 * returns any latched device error. */
aeth_status aeth_get_state(aeth_ctx* ctx, int block, double* cons,
                           double* b1f, double* b2f, double* b3f);

/* The same two copies (Sec. 3.4's set_initial_condition! and the state
 * read after run!), enqueued on the context's stream without waiting, so
 * that a caller with several contexts on several streams overlaps one
 * context's transfers with another's steps.  The host arrays must be
 * page-locked (cudaHostAlloc, cudaHostRegister; AETH_ERR_ARG otherwise):
 * the copy engines move them through the library's device staging buffer
 * (no SM is used for the host link), and a kernel converts between FP64
 * and the working precision.  The caller must not modify the arrays of a
 * set, or read those of a get, before the stream has passed the call
 * (aeth_sync, or a CUDA event recorded after it).  Calls on one context
 * run in stream order; device errors are latched as for aeth_step.
 * b1f..b3f may be NULL in hydro (and, for a get, to skip the field). */
aeth_status aeth_set_state_async(aeth_ctx* ctx, int block, const double* cons,
                                 const double* b1f, const double* b2f,
                                 const double* b3f);
aeth_status aeth_get_state_async(aeth_ctx* ctx, int block, double* cons,
                                 double* b1f, double* b2f, double* b3f);

/* The state of every block in one page-locked host array, block after
 * block in the order of aeth_add_block, each block as cons [5][nz][ny][nx]
 * followed in MHD by b1f, b2f, b3f (the layouts above) and, with dust, by
 * every species' rho_mom [4][nz][ny][nx] (as aeth_set_dust): one copy-engine
 * transfer for the whole mesh instead of four per block, for meshes of
 * many small blocks.  *n receives the array's length in doubles.  The
 * transfers behave as aeth_set_state_async / aeth_get_state_async; the
 * first call allocates a device buffer of that size (AETH_ERR_OOM if it
 * cannot), freed by aeth_destroy. */
aeth_status aeth_state_doubles(aeth_ctx* ctx, size_t* n);
aeth_status aeth_set_state_all_async(aeth_ctx* ctx, const double* packed);
aeth_status aeth_get_state_all_async(aeth_ctx* ctx, double* packed);

/* Dual-energy entropy S = p / rho^(gamma-1) of block `block` (register A,
 * interior cells) into S[nz][ny][nx] (host FP64, caller-owned).  Pinned,
 * mapped host memory is written directly, anything else through the
 * library's staging buffer.  AETH_ERR_STATE when dual energy is off;
 * synchronises the stream. */
aeth_status aeth_get_entropy(aeth_ctx* ctx, int block, double* S);

/* Eq. 11 over every block: dt = C * Cmax * min over cells and directions of
 * dx_d / (|v_d| + c_d), with c_d the directional fast speed (sound speed in
 * hydro, 0 for dust) and Cmax = 1 (VL2, RK2) or 1/(1 + 1/sqrt 2)
 * (IMEX2P).  Synchronises; also leaves dt on the device for
 * aeth_step(ctx, 0). */
aeth_status aeth_compute_dt(aeth_ctx* ctx, double* dt);

/* One cycle of the time integrator (Sec. 2.6: every stage forms the
 * fluxes of Sec. 2.4, the CT update of Sec. 2.5 and the finite-volume
 * update of Eq. 8, combined in the two registers of Eq. 10; the dust runs
 * add the implicit drag of Sec. 2.2): enqueue one full step of length dt on
 * every block.  dt > 0: use it; dt == 0: use the device-resident dt of the
 * last aeth_compute_dt / aeth_run.  Asynchronous; device errors surface at
 * the next synchronising call. */
aeth_status aeth_step(aeth_ctx* ctx, double dt);

/* run! of Sec. 3.4 for a fixed number of cycles: enqueue nsteps steps
 * (Sec. 2.6), each using the CFL step of Eq. 11 computed on the device
 * from the current state after every cycle (no host round trip); the step
 * sequence is captured once into a CUDA graph and replayed.  Asynchronous;
 * AETH_ERR_ARG for nsteps < 0. */
aeth_status aeth_run(aeth_ctx* ctx, int nsteps);

/* End of a run! (Sec. 3.4): wait for the stream and return the latched
 * device status (non-finite state, strict floors, timed-out waits). */
aeth_status aeth_sync(aeth_ctx* ctx);

/* FP64 volume integrals and max relative div B over all blocks (the
 * history quantities of Sec. 3.5).  Synchronises. */
aeth_status aeth_diagnostics(aeth_ctx* ctx, aeth_diag* out);

/* Dust state of species k of a block: rho_mom[4][nz][ny][nx] =
 * (rho_k, M1_k, M2_k, M3_k), host FP64 (Sec. 2.2, Eqs. 6-7). */
aeth_status aeth_set_dust(aeth_ctx* ctx, int block, int k,
                          const double* rho_mom);
aeth_status aeth_get_dust(aeth_ctx* ctx, int block, int k, double* rho_mom);

/* Learned Riemann flux (no counterpart in the paper, which solves every face
 * with HLLD): a 14 -> 128 -> 128 -> 128 -> 7 MLP with SiLU hidden layers.
 * Inputs: the face-frame left/right primitive states and the normal field,
 * made dimensionless with rho_L and c = max(c_f,L, c_f,R): the left state
 * (rho_L = 1 dropped) and Bn, then the jump dW = W_R - W_L on the same
 * scales as d (1 + |dW|) with d = dW / |dW| (its direction at full BF16
 * resolution whatever its size; zero for equal states); zero-padded to 16.
 * Outputs y: the face flux as a correction of the HLLE flux F_E
 * scaled by the jump, F = F_E + k J y, with k the flux scales rho_L c,
 * rho_L c^2 (x3), rho_L c^3 gamma/(gamma-1), sqrt(rho_L) c^2 (x2) and
 * J = (S_R - S_L) (sum_q ((U_R,q - U_L,q) / k_q)^2)^(1/2) the dimensionless
 * jump (Davis speeds S); F tends to the physical flux as the jump vanishes.  Parameter
 * layout (FP32): per layer l, W_l[out][in] row-major then b_l[out]; 52103
 * floats in all.
 *
 * aeth_load_mlp: copy the network to the device (BF16 weights and biases
 * in the layouts of both engines; the library allocates ~160 KB).  With
 * config riemann = AETH_RIEMANN_MLP the step evaluates it on the tensor
 * cores for every face and falls back to HLLD on faces where |F - F_E|
 * exceeds mlp_tau (S_R - S_L) |U_R - U_L| + 2e-2 k in some component, or
 * where the intermediate HLL states F implies lose positive density or
 * pressure; fallbacks are counted in aeth_diag.mlp_fallbacks.  FP32 and
 * FP32_P64 gas runs only. */
aeth_status aeth_load_mlp(aeth_ctx* ctx, const float* params, size_t n);

/* Tensor-core forward pass of the loaded network on n dimensionless feature
 * rows (device d_X [n][16], columns 14 and 15 ignored) into device d_Y
 * [n][8].  Asynchronous on the bound stream.  aeth_mlp_infer: warp
 * mma.sync; aeth_mlp_infer_tc: tcgen05 with TMEM accumulators (d_X, d_Y
 * 16-byte aligned); an MMA wait that runs out latches a status bit that the
 * next synchronising call reports as AETH_ERR_TIMEOUT. */
aeth_status aeth_mlp_infer(aeth_ctx* ctx, const float* d_X, float* d_Y, int n);
aeth_status aeth_mlp_infer_tc(aeth_ctx* ctx, const float* d_X, float* d_Y, int n);

/* The learned face flux on caller-given faces (no counterpart in the paper):
 * the per-face function the flux pass applies under AETH_RIEMANN_MLP --
 * features, the tcgen05 network, F = F_E + k J y, the acceptance checks and
 * the HLLD fallback described at aeth_load_mlp -- on n faces given in the
 * face frame of Sec. 2.4: d_states[n][15] = (rho, vn, vt1, vt2, p, Bt1,
 * Bt2) left, the same right, then Bn (device FP32, caller-owned).  Writes
 * the fluxes d_flux[n][7] = (rho, Mn, Mt1, Mt2, E, Bt1, Bt2) and
 * d_accept[n] (1: the network's flux, 0: HLLD), both device, caller-owned;
 * the fallbacks also count in aeth_diag.mlp_fallbacks.  Asynchronous on the
 * bound stream.  The context must be finalized with the learned flux's
 * configuration (FP32 or FP32_P64 adiabatic gas, its gamma, mlp_tau and
 * MHD or hydro mode) and a loaded network; AETH_ERR_STATE otherwise,
 * AETH_ERR_UNSUPPORTED for FP64, isothermal or dust contexts, AETH_ERR_ARG
 * for n < 0 or NULL arrays. */
aeth_status aeth_mlp_face_flux(aeth_ctx* ctx, const float* d_states, float* d_flux,
                               int* d_accept, int n);

/* Self-test of the bounded device waits (no counterpart in the paper): one
 * warp waits, through the wait the tcgen05 network kernels use, on an
 * mbarrier that never receives an arrival.  The wait gives up after its
 * limit (~0.5 s) and the call returns AETH_ERR_TIMEOUT; the context's own
 * status word is untouched and the context stays usable.  Synchronous;
 * requires aeth_finalize. */
aeth_status aeth_selftest_wait_timeout(aeth_ctx* ctx);

/* Training data from the solver itself: for every stride-th interior cell of
 * every block, the PLM states of its three lower faces (dimensionless
 * features, 16 floats per sample, device array d_X) and the network
 * targets y = (F_HLLD - F_E) / (k J) of their HLLD fluxes (computed in
 * FP64; zero where J < 1e-9; 8 floats per sample, last one zero, d_Y).  At most
 * `capacity` samples are written; *n_out receives the count.  Synchronous.
 * AETH_ERR_UNSUPPORTED for dust runs and for contexts with linked blocks. */
aeth_status aeth_mlp_collect(aeth_ctx* ctx, int stride, float* d_X, float* d_Y,
                             long long capacity, long long* n_out);

/* Training kernels (caller-owned device buffers, enqueued on cuda_stream):
 * aeth_mlp_grad: loss 0.5/n sum |y - t|^2 (device float *d_loss) and its
 * gradient (d_grad, same layout as the parameters) by backpropagation over
 * n samples (d_X [n][16], d_Y [n][8]); d_work holds aeth_mlp_work_floats(n)
 * floats.  aeth_mlp_adam: one Adam update of n parameters (step >= 1). */
aeth_status aeth_mlp_work_floats(int n, size_t* work_floats);
aeth_status aeth_mlp_grad(const float* d_params, const float* d_X,
                          const float* d_Y, int n, float* d_grad, float* d_work,
                          size_t work_floats, float* d_loss, void* cuda_stream);
aeth_status aeth_mlp_adam(float* d_params, const float* d_grad, float* d_m,
                          float* d_v, long long n, int step, float lr,
                          float beta1, float beta2, float eps,
                          void* cuda_stream);

/* Kernel timing for roofline measurements (no counterpart in the paper; the
 * paper times whole cycles only).  enable = 1: every later aeth_step /
 * aeth_run launches its kernels directly (no graph replay) and brackets each
 * launch of the dominant stage kernel with CUDA events on the bound stream.
 * aeth_profile_read synchronises and returns the summed device time (ms) of
 * those launches, their count, and the algorithmic HBM bytes they moved
 * (each launch: its cells x words read and written once x element size).
 * *all_launches counts every kernel the library launched since enable.
 * enable = 0 stops and clears the record. */
aeth_status aeth_profile(aeth_ctx* ctx, int enable);
aeth_status aeth_profile_read(aeth_ctx* ctx, double* total_ms,
                              long long* launches, double* algo_bytes,
                              long long* all_launches);

/* Tile shape of the fused flux pass (no counterpart in the paper): a CTA of
 * 128 threads owns a flux_tx x (128 / flux_tx) column tile of cells and
 * marches kchunk planes along z.  flux_tx = 32 (default), 16, or 0 for band
 * tiles: CTAs of 256 threads over whole rows of a block (its n_x + 2 flux
 * columns), 256 / (n_x + 2) rows at a time, which keep the lanes of blocks
 * narrower than a 2-D tile busy (every block at most 64 cells wide).  16 and 0 are built for FP32
 * and FP32_P64 / FP32_SEL64 contexts with a classical solver, no dual
 * energy, fused path (AETH_ERR_UNSUPPORTED otherwise); kchunk in 1 .. 1024 (the
 * default is the largest of 64, 32, 16, 8, 4 that gives every SM four
 * tiles).  Each face is solved once, by the same code, whatever the shape:
 * the 2-D shapes give identical states, band tiles states within a few
 * FP32 ulps of them (the compiler contracts some multiply-adds of that
 * kernel differently).  aeth_set_flux_tile rebuilds the launch tables
 * (host and device) and drops the captured step graph; call it between
 * steps.  aeth_get_flux_tile reads the current shape. */
aeth_status aeth_set_flux_tile(aeth_ctx* ctx, int flux_tx, int kchunk);
aeth_status aeth_get_flux_tile(aeth_ctx* ctx, int* flux_tx, int* kchunk);

/* Autotuner of the flux pass's tile shape (no counterpart in the paper):
 * times the fused flux pass for z-chunks of 8, 16, 32 and 64 planes per
 * tile, with the 32-wide and (where built) the 16-wide and band tiles, on
 * the current state, and keeps the fastest (written to *flux_tx and
 * *kchunk, either may be NULL).  NOTE: it ADVANCES the state by 3 steps per
 * candidate (up to 36) with the current device dt; call it on a scratch copy or
 * before loading the real state.  The Python helper Solver.tune_tiles
 * keeps each choice in a JSON cache keyed by the block sizes and the
 * configuration. */
aeth_status aeth_autotune(aeth_ctx* ctx, int* flux_tx, int* kchunk);

/* Allocation-free CFL step (the paper has no counterpart: it is a service
 * for callers that may not allocate device memory, e.g. code running inside
 * another framework's caching allocator or a host callback, or under a
 * budget that forbids cudaMalloc after start-up).  Computes the dt of
 * Eq. 11 (ideal-gas closure with the given gamma; no isothermal or
 * dual-energy variant) for ONE Cartesian block whose FP64 state the caller
 * already holds on the device in the host-array layout above (cons[5][nz][ny][nx],
 * b1/b2/b3 face arrays; b* ignored and may be NULL when mhd = 0), with cell
 * widths dx1, dx2, dx3 and Cmax = 1, and writes it to the device double
 * *d_dt on `cuda_stream` (NULL = legacy default stream).  Asynchronous.
 * Allocates nothing: its reduction scratch is a fixed static device array
 * of one double per x-row, so ny * nz must be <= 262144 (2 MiB; every GPU
 * that loads the library keeps it until exit); larger grids are rejected
 * with AETH_ERR_ARG.  A non-finite state makes *d_dt NaN.  The first call
 * on each device looks up that device's scratch address and should happen
 * before any stream capture; with CUDA's lazy module loading (the default)
 * that first call is also when the library's device code, and with it the
 * static array, is loaded onto the device, so it may fail with
 * AETH_ERR_CUDA where no device memory is left: make one call at start-up,
 * after which calls allocate nothing.  The cached address belongs to the
 * device's primary context (the one the CUDA runtime and PyTorch use);
 * callers that switch to another CUcontext on the same device are not
 * supported.  All calls share the scratch: calls that overlap on the GPU
 * (other streams or other host threads) race; serialise them.  Returns
 * AETH_ERR_ARG for bad sizes or pointers, AETH_ERR_CUDA if a launch
 * fails. */
aeth_status aeth_cfl_dt_noalloc(const double* d_cons, const double* d_b1,
                                const double* d_b2, const double* d_b3,
                                int nx, int ny, int nz, double dx1,
                                double dx2, double dx3, double gamma,
                                double rho_floor, double p_floor, double cfl,
                                int mhd, double* d_dt, void* cuda_stream);

/* Measured fused-multiply-add throughput of the current device in FLOP/s
 * (two per FMA) for AETH_FP32 or AETH_FP64: one launch of 8 independent FMA
 * chains per thread over 8 CTAs of 256 threads per SM, timed with CUDA
 * events after a warm-up launch.  The arithmetic roofs for kernels that no
 * HBM or tensor figure bounds.  Synchronises the device; AETH_ERR_ARG for
 * another precision. */
aeth_status aeth_probe_fma(int precision, double* flops_per_s);

/* Reason for the last failure on ctx (static storage inside ctx). */
const char* aeth_last_error(const aeth_ctx* ctx);

/* End of the Simulation's lifetime (Sec. 3.4: the state stays available
 * until the caller lets it go): release device memory the library
 * allocated and the context itself.
 * A bound arena is not freed.  NULL is ignored. */
void aeth_destroy(aeth_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
