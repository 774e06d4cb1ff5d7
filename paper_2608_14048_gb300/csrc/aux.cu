// Ghost fill (Sec. 2.3), host<->device state conversion, the CFL reduction
// of Eq. 11 and the FP64 history diagnostics, for every working precision.
#include <cmath>

#include "runtime.hpp"

namespace aeth {

// ------------------------------------------------------------------------
// block pointers
// ------------------------------------------------------------------------

template <typename R>
BlockPtrs<R> block_ptrs(const aeth_ctx* c, int b) {
  const BlockInfo& B = c->blocks[b];
  BlockPtrs<R> P{};
  P.L = B.L;
  P.tab = (const BlockPtrs<R>*)c->d_tab;
  const long long sz = B.L.size();
  // every array starts on a 256-byte boundary
  const long long pitch = (long long)(array_pitch_bytes(sz, (int)sizeof(R)) / sizeof(R));
  P.pitch = pitch;
  for (int r = 0; r < 2; ++r) {
    R* base = (R*)(c->arena + B.off_reg[r]);
    for (int v = 0; v < NVAR; ++v) P.reg[r][v] = base + v * pitch;
  }
  if (B.off_scratch != (size_t)-1) {
    R* s = (R*)(c->arena + B.off_scratch);
    int q = 0;
    for (int v = 0; v < NPRIM; ++v) P.w[v] = s + (q++) * pitch;
    for (int d = 0; d < 3; ++d)
      for (int v = 0; v < 5; ++v) P.f[d][v] = s + (q++) * pitch;
    for (int d = 0; d < 3; ++d)
      for (int v = 0; v < 2; ++v) P.e[d][v] = s + (q++) * pitch;
    for (int d = 0; d < 3; ++d) P.edge[d] = s + (q++) * pitch;
  }
  if (c->cfg.n_dust > 0) {
    for (int r = 0; r < 2; ++r) P.dust[r] = (R*)(c->arena + B.off_dust[r]);
    P.dflux = (R*)(c->arena + B.off_dflux);
  }
  if (c->cfg.riemann == AETH_RIEMANN_MLP) P.fstate = (R*)(c->arena + B.off_fstate);
  if (is_dual(c))
    for (int r = 0; r < 2; ++r) P.ent[r] = (R*)(c->arena + B.off_ent[r]);
  // geometry tables: 12 separable factors x 3 axes
  const R* t = (const R*)(c->arena + B.off_geo);
  const int g = B.L.g;
  long long ax[3] = {B.L.n[0] + 2 * g + 2, B.L.n[1] + 2 * g + 2, B.L.n[2] + 2 * g + 2};
  long long o = 0;
  auto sep = [&](Sep<R>& s) {
    s.x = t + o; o += ax[0];
    s.y = t + o; o += ax[1];
    s.z = t + o; o += ax[2];
    s.g = g;
  };
  for (int d = 0; d < 3; ++d) sep(P.geo.area[d]);
  sep(P.geo.vol);
  for (int d = 0; d < 3; ++d) sep(P.geo.edge[d]);
  sep(P.geo.invr);
  sep(P.geo.cotr);
  for (int d = 0; d < 3; ++d) sep(P.geo.width[d]);
  return P;
}

template BlockPtrs<float> block_ptrs<float>(const aeth_ctx*, int);
template BlockPtrs<double> block_ptrs<double>(const aeth_ctx*, int);

// Number of R entries in one block's geometry tables.
size_t geometry_len(const Layout& L) {
  return 12ull * (size_t)(L.n[0] + L.n[1] + L.n[2] + 3 * (2 * L.g + 2));
}

// Exact separable factors of Sec. 2.3, computed in FP64 on the host.
template <typename R>
static aeth_status build_geometry_T(aeth_ctx* c) {
  for (size_t b = 0; b < c->blocks.size(); ++b) {
    const BlockInfo& B = c->blocks[b];
    const Layout& L = B.L;
    const int g = L.g;
    const double lo[3] = {B.desc.x1min, B.desc.x2min, B.desc.x3min};
    const double hi[3] = {B.desc.x1max, B.desc.x2max, B.desc.x3max};
    double dx[3];
    for (int d = 0; d < 3; ++d) dx[d] = (hi[d] - lo[d]) / L.n[d];
    std::vector<double> h;
    auto xf = [&](int d, int i) { return lo[d] + i * dx[d]; };
    auto push = [&](int d, auto fn) {
      for (int i = -g; i < L.n[d] + g + 2; ++i) h.push_back(fn(i));
    };
    const bool sph = L.coord == AETH_COORD_SPH;
    auto one = [](int) { return 1.0; };
    if (!sph) {
      auto cst = [&](int d) { return [&, d](int) { return dx[d]; }; };
      // area[0] = dy*dz, area[1] = dx*dz, area[2] = dx*dy
      push(0, one); push(1, cst(1)); push(2, cst(2));
      push(0, cst(0)); push(1, one); push(2, cst(2));
      push(0, cst(0)); push(1, cst(1)); push(2, one);
      push(0, cst(0)); push(1, cst(1)); push(2, cst(2));          // vol
      push(0, cst(0)); push(1, one); push(2, one);                // edge[0]
      push(0, one); push(1, cst(1)); push(2, one);                // edge[1]
      push(0, one); push(1, one); push(2, cst(2));                // edge[2]
      push(0, one); push(1, one); push(2, one);                   // invr (unused)
      push(0, one); push(1, one); push(2, one);                   // cotr (unused)
      push(0, cst(0)); push(1, one); push(2, one);                // width[0]
      push(0, one); push(1, cst(1)); push(2, one);                // width[1]
      push(0, one); push(1, one); push(2, cst(2));                // width[2]
    } else {
      auto r = [&](int i) { return xf(0, i); };
      auto th = [&](int j) { return xf(1, j); };
      const double dphi = dx[2];
      auto dcos = [&](int j) { return cos(th(j)) - cos(th(j + 1)); };
      auto r2f = [&](int i) { return r(i) * r(i); };
      auto hdr2 = [&](int i) { return 0.5 * (r(i + 1) * r(i + 1) - r(i) * r(i)); };
      auto vdr3 = [&](int i) { return (r(i + 1) * r(i + 1) * r(i + 1) - r(i) * r(i) * r(i)) / 3.0; };
      auto cphi = [&](int) { return dphi; };
      // area[0] = r_-^2 (cos th- - cos th+) dphi
      push(0, r2f); push(1, dcos); push(2, cphi);
      // area[1] = 1/2 (r+^2 - r-^2) sin th- dphi
      push(0, hdr2); push(1, [&](int j) { return sin(th(j)); }); push(2, cphi);
      // area[2] = 1/2 (r+^2 - r-^2) (th+ - th-)
      push(0, hdr2); push(1, [&](int) { return dx[1]; }); push(2, one);
      // vol = (r+^3 - r-^3)/3 (cos th- - cos th+) dphi
      push(0, vdr3); push(1, dcos); push(2, cphi);
      // edge[0] = dr ; edge[1] = r_- dth ; edge[2] = r_- sin th- dphi
      push(0, [&](int) { return dx[0]; }); push(1, one); push(2, one);
      push(0, r); push(1, [&](int) { return dx[1]; }); push(2, one);
      push(0, r); push(1, [&](int j) { return sin(th(j)); }); push(2, cphi);
      // <1/r> = (A_r+ - A_r-)/(2V) = (r+^2 - r-^2) / (2 (r+^3 - r-^3)/3)
      push(0, [&](int i) { return (r(i + 1) * r(i + 1) - r(i) * r(i)) / (2.0 * vdr3(i)); });
      push(1, one); push(2, one);
      // <cot th / r> = (A_th+ - A_th-)/V
      push(0, [&](int i) { return hdr2(i) / vdr3(i); });
      push(1, [&](int j) { return (sin(th(j + 1)) - sin(th(j))) / dcos(j); });
      push(2, one);
      // widths at the volume-weighted centroid
      auto rc = [&](int i) {
        double a = r(i), bb = r(i + 1);
        return 0.75 * (pow(bb, 4) - pow(a, 4)) / (pow(bb, 3) - pow(a, 3));
      };
      auto thc = [&](int j) {
        double a = th(j), bb = th(j + 1);
        return (sin(bb) - sin(a) - bb * cos(bb) + a * cos(a)) / (cos(a) - cos(bb));
      };
      push(0, [&](int) { return dx[0]; }); push(1, one); push(2, one);
      push(0, rc); push(1, [&](int) { return dx[1]; }); push(2, one);
      push(0, rc); push(1, [&](int j) { return sin(thc(j)); }); push(2, cphi);
    }
    if (h.size() != B.geo_len)
      return fail(c, AETH_ERR_STATE, "geometry table size mismatch (%zu vs %zu)", h.size(), B.geo_len);
    std::vector<R> hr(h.begin(), h.end());
    AETH_CK(c, cudaMemcpyAsync(c->arena + B.off_geo, hr.data(), hr.size() * sizeof(R),
                               cudaMemcpyHostToDevice, c->stream));
    AETH_CK(c, cudaStreamSynchronize(c->stream));
  }
  return AETH_OK;
}

aeth_status build_geometry(aeth_ctx* c) {
  return c->elem == 8 ? build_geometry_T<double>(c) : build_geometry_T<float>(c);
}

// Device block table and the tile prefix sums of every pass kind.
// Default z extent of a flux tile: the largest of {64, 32, 16, 8, 4} that
// still gives every SM at least four tiles (small grids need short
// chunks to fill the GPU; long chunks amortise the z-halo warm-up).
static int default_kchunk(const aeth_ctx* c) {
  const int want = 4 * c->num_sms;
  for (int kc : {64, 32, 16, 8, 4}) {
    long long tiles = 0;
    for (const auto& B : c->blocks) tiles += tiles_of(B.L, PK_FLUX, kc, c->flux_tx);
    if (tiles >= want) return kc;
  }
  return 4;
}

template <typename R>
static aeth_status build_tables_T(aeth_ctx* c) {
  const int nb = (int)c->blocks.size();
  if (c->kchunk <= 0) c->kchunk = default_kchunk(c);
  std::vector<BlockPtrs<R>> tab(nb);
  for (int b = 0; b < nb; ++b) tab[b] = block_ptrs<R>(c, b);
  c->h_prefix.assign((size_t)PK_N * (nb + 1), 0);
  for (int kind = 0; kind < PK_N; ++kind) {
    int* p = c->h_prefix.data() + kind * (nb + 1);
    long long acc = 0;
    for (int b = 0; b < nb; ++b) {
      p[b] = (int)acc;
      acc += tiles_of(c->blocks[b].L, kind, c->kchunk, c->flux_tx);
    }
    if (acc > (1ll << 30)) return fail(c, AETH_ERR_ARG, "too many tiles (%lld)", acc);
    p[nb] = (int)acc;
  }
  AETH_CK(c, cudaMemcpyAsync(c->d_tab, tab.data(), nb * sizeof(BlockPtrs<R>),
                             cudaMemcpyHostToDevice, c->stream));
  AETH_CK(c, cudaMemcpyAsync(c->d_prefix, c->h_prefix.data(), c->h_prefix.size() * sizeof(int),
                             cudaMemcpyHostToDevice, c->stream));
  std::vector<int2> maps[PK_N];
  for (int kind = 0; kind < PK_N; ++kind) {
    if (!c->d_tmap[kind]) continue;
    const int* p = c->h_prefix.data() + kind * (nb + 1);
    if (p[nb] != c->tmap_n[kind]) return fail(c, AETH_ERR_STATE, "tile map size mismatch");
    maps[kind].resize((size_t)p[nb]);
    for (int b = 0; b < nb; ++b)
      for (int t = p[b]; t < p[b + 1]; ++t) maps[kind][t] = make_int2(b, t - p[b]);
    AETH_CK(c, cudaMemcpyAsync(c->d_tmap[kind], maps[kind].data(), maps[kind].size() * sizeof(int2),
                               cudaMemcpyHostToDevice, c->stream));
  }
  AETH_CK(c, cudaStreamSynchronize(c->stream));
  return AETH_OK;
}

aeth_status build_tables(aeth_ctx* c) {
  return c->elem == 8 ? build_tables_T<double>(c) : build_tables_T<float>(c);
}

// ------------------------------------------------------------------------
// ghost fill, one axis at a time (edges and corners come out right)
// ------------------------------------------------------------------------

template <typename R>
__global__ void k_fill_axis(Layout L, Arr8<R> a, int nv, int d) {
  const int g = L.g;
  int lo[3], ext[3];
  for (int e = 0; e < 3; ++e) {
    if (e < d) { lo[e] = -g; ext[e] = L.n[e] + 2 * g + 1; }
    else if (e == d) { lo[e] = 0; ext[e] = 2 * g + 1; }
    else { lo[e] = 0; ext[e] = L.n[e] + 1; }
  }
  const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
  const int t1 = blockIdx.y * blockDim.y + threadIdx.y;
  const int t2 = blockIdx.z * blockDim.z + threadIdx.z;
  if (t0 >= ext[0] || t1 >= ext[1] || t2 >= ext[2]) return;
  int c[3] = {t0 + lo[0], t1 + lo[1], t2 + lo[2]};
  const int n = L.n[d];
  const int t = c[d];
  c[d] = t < g ? t - g : n + (t - g);      // -g..-1, n..n+g
  const int p = c[d];
  const long long dst = L.idx(c[0], c[1], c[2]);
  // every source loaded before the first store: the stores go through the
  // same arrays, so interleaving them would serialise the round trips
  R val[NVAR];
  bool on[NVAR];
#pragma unroll
  for (int v = 0; v < NVAR; ++v) {
    on[v] = false;
    if (v >= nv) continue;
    const bool face_d = (v == 5 + d);
    int s;
    if (L.bc[d] == AETH_BC_PERIODIC) {
      s = ((p % n) + n) % n;
    } else if (face_d) {
      if (p >= 0 && p <= n) continue;       // faces 0..n are real
      s = p < 0 ? 0 : n;
    } else {
      s = p < 0 ? 0 : n - 1;
    }
    int sc[3] = {c[0], c[1], c[2]};
    sc[d] = s;
    val[v] = a.p[v][L.idx(sc[0], sc[1], sc[2])];
    on[v] = true;
  }
#pragma unroll
  for (int v = 0; v < NVAR; ++v)
    if (on[v]) a.p[v][dst] = val[v];
}

template <typename R>
void launch_fill(const BlockPtrs<R>& P, R* const* arrs, int nv, cudaStream_t st) {
  Arr8<R> a{};
  for (int v = 0; v < nv; ++v) a.p[v] = arrs[v];
  const Layout& L = P.L;
  for (int d = 0; d < 3; ++d) {
    int ext[3];
    for (int e = 0; e < 3; ++e)
      ext[e] = e < d ? L.n[e] + 2 * L.g + 1 : (e == d ? 2 * L.g + 1 : L.n[e] + 1);
    dim3 blk(32, 4, 2);
    dim3 grd((ext[0] + 31) / 32, (ext[1] + 3) / 4, (ext[2] + 1) / 2);
    k_fill_axis<R><<<grd, blk, 0, st>>>(L, a, nv, d);
  }
}
template void launch_fill<float>(const BlockPtrs<float>&, float* const*, int, cudaStream_t);
template void launch_fill<double>(const BlockPtrs<double>&, double* const*, int, cudaStream_t);

// ------------------------------------------------------------------------
// host FP64 <-> device working precision (interior only)
// ------------------------------------------------------------------------

// Dual energy (ent != null): the entropy S = p / rho^(gamma-1) of each
// interior cell from the FP64 input (p from E with the floors of Eq. 5).
struct DualInit {
  double gamma, rho_floor, p_floor;
};

template <typename R>
__global__ void k_load(Layout L, Arr8<R> a, int mhd, const double* __restrict__ sc,
                       const double* __restrict__ b1, const double* __restrict__ b2,
                       const double* __restrict__ b3, R* __restrict__ ent, DualInit di) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z * blockDim.z + threadIdx.z;
  const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
  if (i > nx || j > ny || k > nz) return;
  const long long nc = (long long)nx * ny * nz;
  const long long d = L.idx(i, j, k);
  if (i < nx && j < ny && k < nz) {
    const long long c = ((long long)k * ny + j) * nx + i;
    for (int v = 0; v < 5; ++v) a.p[v][d] = (R)sc[v * nc + c];
    if (ent) {
      const double rho = fmax(sc[c], di.rho_floor);
      const double m1 = sc[nc + c], m2 = sc[2 * nc + c], m3 = sc[3 * nc + c];
      double km = 0.5 * (m1 * m1 + m2 * m2 + m3 * m3) / rho;
      if (mhd) {
        const double x = 0.5 * (b1[((long long)k * ny + j) * (nx + 1) + i] +
                                b1[((long long)k * ny + j) * (nx + 1) + i + 1]);
        const double y = 0.5 * (b2[((long long)k * (ny + 1) + j) * nx + i] +
                                b2[((long long)k * (ny + 1) + j + 1) * nx + i]);
        const double z = 0.5 * (b3[((long long)k * ny + j) * nx + i] +
                                b3[((long long)(k + 1) * ny + j) * nx + i]);
        km += 0.5 * (x * x + y * y + z * z);
      }
      const double pr = fmax((di.gamma - 1.0) * (sc[4 * nc + c] - km), di.p_floor);
      ent[d] = (R)(pr / pow(rho, di.gamma - 1.0));
    }
  }
  if (!mhd) return;
  if (j < ny && k < nz) a.p[5][d] = (R)b1[((long long)k * ny + j) * (nx + 1) + i];
  if (i < nx && k < nz) a.p[6][d] = (R)b2[((long long)k * (ny + 1) + j) * nx + i];
  if (i < nx && j < ny) a.p[7][d] = (R)b3[((long long)k * ny + j) * nx + i];
}

template <typename R>
__global__ void k_store(Layout L, Arr8<R> a, int mhd, double* __restrict__ sc,
                        double* __restrict__ b1, double* __restrict__ b2, double* __restrict__ b3) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z * blockDim.z + threadIdx.z;
  const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
  if (i > nx || j > ny || k > nz) return;
  const long long nc = (long long)nx * ny * nz;
  if (i < nx && j < ny && k < nz) {
    const long long c = ((long long)k * ny + j) * nx + i;
    const long long d = L.idx(i, j, k);
    for (int v = 0; v < 5; ++v) sc[v * nc + c] = (double)a.p[v][d];
  }
  if (!mhd) return;
  // periodic axes: the last face is the image of the first
  // (a linked high side keeps its face n current: the neighbour's update
  // writes it)
  const int i1 = (i == nx && L.bc[0] == AETH_BC_PERIODIC && L.lnk[0][1] < 0) ? 0 : i;
  const int j2 = (j == ny && L.bc[1] == AETH_BC_PERIODIC && L.lnk[1][1] < 0) ? 0 : j;
  const int k3 = (k == nz && L.bc[2] == AETH_BC_PERIODIC && L.lnk[2][1] < 0) ? 0 : k;
  if (j < ny && k < nz) b1[((long long)k * ny + j) * (nx + 1) + i] = (double)a.p[5][L.idx(i1, j, k)];
  if (i < nx && k < nz) b2[((long long)k * (ny + 1) + j) * nx + i] = (double)a.p[6][L.idx(i, j2, k)];
  if (i < nx && j < ny) b3[((long long)k * ny + j) * nx + i] = (double)a.p[7][L.idx(i, j, k3)];
}

template <typename R>
static aeth_status load_store_T(aeth_ctx* c, int b, bool load, double* const* io) {
  BlockPtrs<R> P = block_ptrs<R>(c, b);
  Arr8<R> a{};
  for (int v = 0; v < NVAR; ++v) a.p[v] = P.reg[0][v];
  const Layout& L = P.L;
  dim3 blk(32, 4, 2);
  dim3 grd((L.n[0] + 1 + 31) / 32, (L.n[1] + 1 + 3) / 4, (L.n[2] + 1 + 1) / 2);
  const DualInit di{c->cfg.gamma, c->cfg.rho_floor, c->cfg.p_floor};
  if (load)
    k_load<R><<<grd, blk, 0, c->stream>>>(L, a, is_mhd(c), io[0], io[1], io[2], io[3], P.ent[0],
                                          di);
  else k_store<R><<<grd, blk, 0, c->stream>>>(L, a, is_mhd(c), io[0], io[1], io[2], io[3]);
  AETH_CK(c, cudaGetLastError());
  return AETH_OK;
}

aeth_status enqueue_load(aeth_ctx* c, int b, double* const* io) {
  return c->elem == 8 ? load_store_T<double>(c, b, true, io) : load_store_T<float>(c, b, true, io);
}
aeth_status enqueue_store(aeth_ctx* c, int b, double* const* io) {
  return c->elem == 8 ? load_store_T<double>(c, b, false, io) : load_store_T<float>(c, b, false, io);
}

// dust species k: rho_mom[4][nz][ny][nx] <-> register A
template <typename R>
__global__ void k_dust_io(Layout L, R* __restrict__ dreg, int k, int load,
                          double* __restrict__ s) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int kk = blockIdx.z * blockDim.z + threadIdx.z;
  const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
  if (i >= nx || j >= ny || kk >= nz) return;
  const long long nc = (long long)nx * ny * nz;
  const long long c = ((long long)kk * ny + j) * nx + i;
  const long long d = L.idx(i, j, kk);
  const long long sz = L.size();
  for (int v = 0; v < 4; ++v) {
    R* arr = dreg + (long long)(4 * k + v) * sz;
    if (load) arr[d] = (R)s[v * nc + c];
    else s[v * nc + c] = (double)arr[d];
  }
}

template <typename R>
static aeth_status dust_io_T(aeth_ctx* c, int b, int k, bool load, double* io) {
  BlockPtrs<R> P = block_ptrs<R>(c, b);
  const Layout& L = P.L;
  dim3 blk(32, 4, 2);
  dim3 grd((L.n[0] + 31) / 32, (L.n[1] + 3) / 4, (L.n[2] + 1) / 2);
  k_dust_io<R><<<grd, blk, 0, c->stream>>>(L, P.dust[0], k, load ? 1 : 0, io);
  AETH_CK(c, cudaGetLastError());
  return AETH_OK;
}
// dual-energy entropy of register A (interior) -> S[nz][ny][nx]
template <typename R>
__global__ void k_entropy_store(Layout L, const R* __restrict__ ent, double* __restrict__ s) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z * blockDim.z + threadIdx.z;
  const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
  if (i >= nx || j >= ny || k >= nz) return;
  s[((long long)k * ny + j) * nx + i] = (double)ent[L.idx(i, j, k)];
}

template <typename R>
static aeth_status entropy_store_T(aeth_ctx* c, int b, double* io) {
  BlockPtrs<R> P = block_ptrs<R>(c, b);
  const Layout& L = P.L;
  dim3 blk(32, 4, 2);
  dim3 grd((L.n[0] + 31) / 32, (L.n[1] + 3) / 4, (L.n[2] + 1) / 2);
  k_entropy_store<R><<<grd, blk, 0, c->stream>>>(L, P.ent[0], io);
  AETH_CK(c, cudaGetLastError());
  return AETH_OK;
}
aeth_status enqueue_entropy_store(aeth_ctx* c, int b, double* io) {
  return c->elem == 8 ? entropy_store_T<double>(c, b, io) : entropy_store_T<float>(c, b, io);
}

aeth_status enqueue_dust_load(aeth_ctx* c, int b, int k, double* io) {
  return c->elem == 8 ? dust_io_T<double>(c, b, k, true, io) : dust_io_T<float>(c, b, k, true, io);
}
aeth_status enqueue_dust_store(aeth_ctx* c, int b, int k, double* io) {
  return c->elem == 8 ? dust_io_T<double>(c, b, k, false, io) : dust_io_T<float>(c, b, k, false, io);
}

// ------------------------------------------------------------------------
// CFL reduction (Eq. 11): per-cell min over directions, block min, then one
// block reduces all partials.  Non-finite states latch ST_NONFINITE.
// ------------------------------------------------------------------------

__device__ __forceinline__ double warp_min(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// CFL time step (Eq. 11) over all blocks: one partial minimum per CTA.  The
// work unit is the 32x4x2 cell tile of the elementwise passes (full warps
// on every block size, one block lookup per 256 cells); a CTA iteration
// takes TPI tiles and loads all of them before using any, so each thread
// keeps TPI independent load groups in flight.
// DUAL: dual energy, the pressure of an untrusted internal energy comes
// from the entropy (Sec. 2.8)
template <typename R, bool P64, typename Src, bool DUAL = false>
__global__ void __launch_bounds__(256)
    k_dt(Src S, int total, int mhd, double gamma, double rho_floor, double p_floor, int nd,
         double cs2, double alpha_switch, float p64_ratio, double* __restrict__ partial,
         int* status) {
  constexpr bool dual = DUAL;
  // cs2 > 0: isothermal closure p = cs2 rho, fast speed with gamma = 1
  const bool iso = cs2 > 0.0;
  constexpr int TPI = 2;
  __shared__ double sm[8];
  R m = R(INFINITY);   // running minimum in the working precision
  bool bad = false;
  const int tx = (int)threadIdx.x % CELL_BX, ty = ((int)threadIdx.x / CELL_BX) % CELL_BY;
  const int tz = (int)threadIdx.x / (CELL_BX * CELL_BY);
  for (int t0 = blockIdx.x * TPI; t0 < total; t0 += gridDim.x * TPI) {
    R a[TPI][5], bf[TPI][6], wd[TPI][3], sv[TPI];
    int ci[TPI][3];
    bool on[TPI];
#pragma unroll
    for (int q = 0; q < TPI; ++q) {
      on[q] = false;
      const int t = t0 + q;
      if (t >= total) continue;
      int loc;
      const BlockPtrs<R>& P = S.get(t, loc);
      const Layout L = P.L;
      const int ntx = (L.n[0] + CELL_BX) / CELL_BX, nty = (L.n[1] + CELL_BY) / CELL_BY;
      const int i = (loc % ntx) * CELL_BX + tx, j = ((loc / ntx) % nty) * CELL_BY + ty;
      const int k = (loc / (ntx * nty)) * CELL_BZ + tz;
      if (i >= L.n[0] || j >= L.n[1] || k >= L.n[2]) continue;
      on[q] = true;
      ci[q][0] = i; ci[q][1] = j; ci[q][2] = k;
      const long long c = L.idx(i, j, k);
      const R* const* u = P.reg[0];
#pragma unroll
      for (int v = 0; v < 5; ++v) a[q][v] = (v == 4 && iso) ? R(0) : u[v][c];   // no energy
      if constexpr (DUAL) sv[q] = P.ent[0][c];
      if (mhd) {
        bf[q][0] = u[5][c]; bf[q][1] = u[5][c + 1];
        bf[q][2] = u[6][c]; bf[q][3] = u[6][c + L.sx];
        bf[q][4] = u[7][c]; bf[q][5] = u[7][c + L.sx * L.sy];
      }
#pragma unroll
      for (int d = 0; d < 3; ++d) wd[q][d] = P.geo.width[d](i, j, k);
    }
#pragma unroll
    for (int q = 0; q < TPI; ++q) {
      if (!on[q]) continue;
      R rho = a[q][0];
      if (!(rho >= (R)rho_floor)) { if (!(rho == rho)) bad = true; rho = (R)rho_floor; }
      const R v[3] = {a[q][1] / rho, a[q][2] / rho, a[q][3] / rho};
      R bc[3] = {0, 0, 0};
      if (mhd) {
        bc[0] = R(0.5) * (bf[q][0] + bf[q][1]);
        bc[1] = R(0.5) * (bf[q][2] + bf[q][3]);
        bc[2] = R(0.5) * (bf[q][4] + bf[q][5]);
      }
      R pr;
      if (iso) {
        pr = (R)cs2 * rho;
      } else if constexpr (DUAL) {
        const R ke = R(0.5) * rho * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        const R me = R(0.5) * (bc[0] * bc[0] + bc[1] * bc[1] + bc[2] * bc[2]);
        const R eint = a[q][4] - ke - me;
        pr = eint < (R)alpha_switch * (ke + me) ? sv[q] * pow(rho, (R)(gamma - 1.0))
                                                : (R)(gamma - 1.0) * eint;
      } else if (P64) {
        // FP64 subtraction in every cell, or only where the FP32 one cancels
        bool wide = true;
        if (p64_ratio > 0.0f) {
          const R ke = R(0.5) * rho * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
          const R me = R(0.5) * (bc[0] * bc[0] + bc[1] * bc[1] + bc[2] * bc[2]);
          const R ei = a[q][4] - ke - me;
          wide = ke + me > (R)p64_ratio * ei;
          pr = (R)(gamma - 1.0) * ei;
        }
        if (wide) {
          double ke = 0.5 * ((double)a[q][1] * a[q][1] + (double)a[q][2] * a[q][2] +
                             (double)a[q][3] * a[q][3]) / (double)rho;
          double me = 0.5 * ((double)bc[0] * bc[0] + (double)bc[1] * bc[1] + (double)bc[2] * bc[2]);
          pr = (R)((gamma - 1.0) * ((double)a[q][4] - ke - me));
        }
      } else {
        pr = (R)(gamma - 1.0) * (a[q][4] - R(0.5) * rho * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) -
                                 R(0.5) * (bc[0] * bc[0] + bc[1] * bc[1] + bc[2] * bc[2]));
      }
      if (!(pr >= (R)p_floor)) { if (!(pr == pr)) bad = true; pr = (R)p_floor; }
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const R cf = fast_speed(iso ? R(1) : (R)gamma, rho, pr, bc[d], bc[(d + 1) % 3],
                                bc[(d + 2) % 3]);
        const R dtd = wd[q][d] / (fabs(v[d]) + cf);
        if (!(dtd > R(0))) bad = true;
        m = fmin(m, dtd);
      }
      // pressureless dust species: c = 0 (Eq. 11)
      if (nd > 0) {
        int loc;
        const BlockPtrs<R>& P = S.get(t0 + q, loc);
        const Layout L = P.L;
        const long long c = L.idx(ci[q][0], ci[q][1], ci[q][2]);
        const long long sz = L.size();
        for (int sp = 0; sp < nd; ++sp) {
          const R rk = P.dust[0][(long long)(4 * sp) * sz + c];
          if (!(rk > R(0))) continue;
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            const R vk = fabs(P.dust[0][(long long)(4 * sp + 1 + d) * sz + c] / rk);
            if (vk > R(0)) m = fmin(m, wd[q][d] / vk);
          }
        }
      }
    }
  }
  const double md = warp_min((double)m);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = md;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : INFINITY;
    v = warp_min(v);
    if (threadIdx.x == 0) partial[blockIdx.x] = v;
  }
  if (bad) atomicOr(status, ST_NONFINITE);
}

// 0: the one-cell-per-thread CFL pass everywhere
#ifndef AETH_DT_V4
#define AETH_DT_V4 1
#endif

// The same CFL step for FP32 gas without dual energy or dust, four
// consecutive x cells per thread: 16-byte loads of the state (the x-face
// field's fifth face as one scalar), the per-cell arithmetic of k_dt.  A
// CTA of 256 threads takes four 32 x 4 x 2 cell tiles per iteration.  A
// group of four cells that is not whole inside the block (the x end of the
// row) is done cell by cell.
__device__ __forceinline__ float4 ld4c(const float* p) {
  return *reinterpret_cast<const float4*>(p);
}
__device__ __forceinline__ float el4(const float4& v, int q) {
  return q == 0 ? v.x : (q == 1 ? v.y : (q == 2 ? v.z : v.w));
}

template <bool P64, typename Src>
__global__ void __launch_bounds__(256)
    k_dt_v4(Src S, int total, int mhd, float gamma, float rho_floor, float p_floor, float cs2,
            float p64_ratio, double* __restrict__ partial, int* status) {
  __shared__ double sm[8];
  const bool iso = cs2 > 0.0f;
  float m = INFINITY;
  bool bad = false;
  const int lt = (int)threadIdx.x & 63, sub = (int)threadIdx.x >> 6;
  const int tx4 = 4 * (lt % (CELL_BX / 4)), ty = (lt / (CELL_BX / 4)) % CELL_BY;
  const int tz = lt / ((CELL_BX / 4) * CELL_BY);
  // one cell's Eq. 11 term: min over directions of width / (|v| + c_f)
  auto cell = [&](float rho, float m1, float m2, float m3, float e, const float* bc,
                  const float* wd) {
    if (!(rho >= rho_floor)) { if (!(rho == rho)) bad = true; rho = rho_floor; }
    const float v[3] = {m1 / rho, m2 / rho, m3 / rho};
    float pr;
    if (iso) {
      pr = cs2 * rho;
    } else {
      const float ke = 0.5f * rho * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
      const float me = 0.5f * (bc[0] * bc[0] + bc[1] * bc[1] + bc[2] * bc[2]);
      bool wide = P64;
      if (P64 && p64_ratio > 0.0f) {
        const float ei = e - ke - me;
        wide = ke + me > p64_ratio * ei;
        pr = (gamma - 1.0f) * ei;
      }
      if (wide) {
        const double ked = 0.5 * ((double)m1 * m1 + (double)m2 * m2 + (double)m3 * m3) / (double)rho;
        const double med = 0.5 * ((double)bc[0] * bc[0] + (double)bc[1] * bc[1] +
                                  (double)bc[2] * bc[2]);
        pr = (float)(((double)gamma - 1.0) * ((double)e - ked - med));
      } else if (!P64) {
        pr = (gamma - 1.0f) * (e - ke - me);
      }
    }
    if (!(pr >= p_floor)) { if (!(pr == pr)) bad = true; pr = p_floor; }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const float cf = fast_speed(iso ? 1.0f : gamma, rho, pr, bc[d], bc[(d + 1) % 3],
                                  bc[(d + 2) % 3]);
      const float dtd = wd[d] / (fabsf(v[d]) + cf);
      if (!(dtd > 0.0f)) bad = true;
      m = fminf(m, dtd);
    }
  };
  for (int t = blockIdx.x * 4 + sub; t < total; t += gridDim.x * 4) {
    int loc;
    const BlockPtrs<float>& P = S.get(t, loc);
    const Layout& L = P.L;
    const int ntx = (L.n[0] + CELL_BX) / CELL_BX, nty = (L.n[1] + CELL_BY) / CELL_BY;
    const int i4 = (loc % ntx) * CELL_BX + tx4, j = ((loc / ntx) % nty) * CELL_BY + ty;
    const int k = (loc / (ntx * nty)) * CELL_BZ + tz;
    if (i4 >= L.n[0] || j >= L.n[1] || k >= L.n[2]) continue;
    const long long c = L.idx(i4, j, k);
    const float* const* u = P.reg[0];
    if (i4 + 3 >= L.n[0]) {
      for (int q = 0; i4 + q < L.n[0]; ++q) {
        const long long cq = c + q;
        float bc[3] = {0.0f, 0.0f, 0.0f};
        if (mhd) {
          bc[0] = 0.5f * (u[5][cq] + u[5][cq + 1]);
          bc[1] = 0.5f * (u[6][cq] + u[6][cq + L.sx]);
          bc[2] = 0.5f * (u[7][cq] + u[7][cq + L.sx * L.sy]);
        }
        const float wd[3] = {P.geo.width[0](i4 + q, j, k), P.geo.width[1](i4 + q, j, k),
                             P.geo.width[2](i4 + q, j, k)};
        cell(u[0][cq], u[1][cq], u[2][cq], u[3][cq], iso ? 0.0f : u[4][cq], bc, wd);
      }
      continue;
    }
    const float4 r4 = ld4c(u[0] + c), a4 = ld4c(u[1] + c), b4 = ld4c(u[2] + c),
                 c4 = ld4c(u[3] + c);
    const float4 e4 = iso ? make_float4(0.f, 0.f, 0.f, 0.f) : ld4c(u[4] + c);
    float4 x0 = make_float4(0.f, 0.f, 0.f, 0.f), y0 = x0, y1 = x0, z0 = x0, z1 = x0;
    float x4 = 0.0f;
    if (mhd) {
      x0 = ld4c(u[5] + c);
      x4 = u[5][c + 4];
      y0 = ld4c(u[6] + c);
      y1 = ld4c(u[6] + c + L.sx);
      z0 = ld4c(u[7] + c);
      z1 = ld4c(u[7] + c + L.sx * L.sy);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float xp = q < 3 ? el4(x0, q + 1) : x4;
      const float bc[3] = {0.5f * (el4(x0, q) + xp), 0.5f * (el4(y0, q) + el4(y1, q)),
                           0.5f * (el4(z0, q) + el4(z1, q))};
      const float wd[3] = {P.geo.width[0](i4 + q, j, k), P.geo.width[1](i4 + q, j, k),
                           P.geo.width[2](i4 + q, j, k)};
      cell(el4(r4, q), el4(a4, q), el4(b4, q), el4(c4, q), el4(e4, q), bc, wd);
    }
  }
  const double md = warp_min((double)m);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = md;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : INFINITY;
    v = warp_min(v);
    if (threadIdx.x == 0) partial[blockIdx.x] = v;
  }
  if (bad) atomicOr(status, ST_NONFINITE);
}

__global__ void k_dt_final(const double* __restrict__ partial, int n, double scale,
                           double* __restrict__ dt) {
  __shared__ double sm[32];
  double m = INFINITY;
  for (int t = threadIdx.x; t < n; t += blockDim.x) m = fmin(m, partial[t]);
  m = warp_min(m);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : INFINITY;
    v = warp_min(v);
    if (threadIdx.x == 0) *dt = scale * v;
  }
}

template <typename R, bool P64>
static aeth_status dt_T(aeth_ctx* c) {
  const int nb = (int)c->blocks.size();
  const int total = prefix_total(c, PK_CELL);
  // 2 tiles per CTA iteration; at most dt_grid partial minima
  const int grid = std::max(1, std::min(c->dt_grid, (total + 1) / 2));
  const double cs2 = is_iso(c) ? c->cfg.cs_iso * c->cfg.cs_iso : 0.0;
  const double dual_a = is_dual(c) ? c->cfg.alpha_switch : 0.0;
  // returns the number of partial minima written
  auto launch = [&](auto src) -> int {
    using Src = decltype(src);
    if constexpr (sizeof(R) == 4) {
      if (dual_a <= 0.0 && c->cfg.n_dust == 0 && AETH_DT_V4) {
        // FP32 gas: four x cells per thread
        const int g4 = std::max(1, std::min(c->dt_grid, (total + 3) / 4));
        k_dt_v4<P64, Src><<<g4, 256, 0, c->stream>>>(
            src, total, is_mhd(c), (float)c->cfg.gamma, (float)c->cfg.rho_floor,
            (float)c->cfg.p_floor, (float)cs2,
            c->cfg.precision == AETH_FP32_SEL64 ? (float)c->cfg.p64_ratio : 0.0f, c->d_partials,
            c->d_status);
        return g4;
      }
    }
    auto kernel = dual_a > 0.0 ? k_dt<R, P64, Src, true> : k_dt<R, P64, Src, false>;
    kernel<<<grid, 256, 0, c->stream>>>(src, total, is_mhd(c), c->cfg.gamma, c->cfg.rho_floor,
                                         c->cfg.p_floor, c->cfg.n_dust, cs2, dual_a,
                                         c->cfg.precision == AETH_FP32_SEL64
                                             ? (float)c->cfg.p64_ratio : 0.0f,
                                         c->d_partials, c->d_status);
    return grid;
  };
  int nparts;
  if (nb == 1) {
    nparts = launch(ParamSrc<R>{block_ptrs<R>(c, 0), 0});
  } else {
    nparts = launch(TableSrc<R>{(const BlockPtrs<R>*)c->d_tab, c->d_prefix + PK_CELL * (nb + 1),
                                nb, c->d_tmap[PK_CELL]});
  }
  c->n_launch += 2;
  const double scale = c->cfg.cfl * cmax_of(c->cfg.integrator);
  k_dt_final<<<1, 1024, 0, c->stream>>>(c->d_partials, nparts, scale, c->d_dt);
  AETH_CK(c, cudaGetLastError());
  return AETH_OK;
}

aeth_status enqueue_dt(aeth_ctx* c) {
  if (c->cfg.precision == AETH_FP64) return dt_T<double, false>(c);
  if (c->cfg.precision == AETH_FP32) return dt_T<float, false>(c);
  return dt_T<float, true>(c);
}

__global__ void k_set_dt(double* d, double v) { *d = v; }

aeth_status enqueue_set_dt(aeth_ctx* c, double dt) {
  k_set_dt<<<1, 1, 0, c->stream>>>(c->d_dt, dt);
  c->n_launch += 1;
  AETH_CK(c, cudaGetLastError());
  return AETH_OK;
}

// ------------------------------------------------------------------------
// diagnostics: FP64 volume integrals and max relative div B
// ------------------------------------------------------------------------

template <typename R>
__global__ void __launch_bounds__(256)
    k_diag(const BlockPtrs<R>* __restrict__ tab, const int* __restrict__ pre, int nb, int total,
           int mhd, double* __restrict__ partial) {
  __shared__ double sm[6][8];
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int t = blockIdx.x; t < total; t += gridDim.x) {
    const int b = find_block(pre, nb, t);
    const BlockPtrs<R>& P = tab[b];
    const Layout L = P.L;
    const int r = t - pre[b];
    const int j = r % L.n[1], k = r / L.n[1];
    const R* const* a = P.reg[0];
    for (int i = threadIdx.x; i < L.n[0]; i += blockDim.x) {
      const long long c = L.idx(i, j, k);
      const double V = (double)P.geo.vol(i, j, k);
      for (int v = 0; v < 5; ++v) acc[v] += (double)a[v][c] * V;
      if (mhd) {
        const double f[6] = {a[5][c], a[5][c + 1], a[6][c], a[6][c + L.sx],
                             a[7][c], a[7][c + L.sx * L.sy]};
        const double ar[6] = {P.geo.area[0](i, j, k), P.geo.area[0](i + 1, j, k),
                              P.geo.area[1](i, j, k), P.geo.area[1](i, j + 1, k),
                              P.geo.area[2](i, j, k), P.geo.area[2](i, j, k + 1)};
        const double div = ar[1] * f[1] - ar[0] * f[0] + ar[3] * f[3] - ar[2] * f[2] +
                           ar[5] * f[5] - ar[4] * f[4];
        double den = 0;
        for (int q = 0; q < 6; ++q) den += ar[q] * fabs(f[q]);
        if (den > 0) acc[5] = fmax(acc[5], fabs(div) / den);
      }
    }
  }
  for (int q = 0; q < 5; ++q) acc[q] = warp_sum(acc[q]);
  for (int o = 16; o > 0; o >>= 1) acc[5] = fmax(acc[5], __shfl_xor_sync(0xffffffffu, acc[5], o));
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0)
    for (int q = 0; q < 6; ++q) sm[q][w] = acc[q];
  __syncthreads();
  if (threadIdx.x < 32) {
    const int nw = blockDim.x >> 5;
    for (int q = 0; q < 6; ++q) {
      double v = threadIdx.x < nw ? sm[q][threadIdx.x] : 0.0;
      if (q < 5) v = warp_sum(v);
      else for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
      if (threadIdx.x == 0) partial[6 * blockIdx.x + q] = v;
    }
  }
}

__global__ void k_diag_final(const double* __restrict__ partial, int n, double* out) {
  // fixed assignment of partials to threads and a fixed reduction tree:
  // deterministic totals
  __shared__ double sm[6][256];
  double s[6] = {0, 0, 0, 0, 0, 0};
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    for (int q = 0; q < 5; ++q) s[q] += partial[6 * t + q];
    s[5] = fmax(s[5], partial[6 * t + 5]);
  }
  for (int q = 0; q < 6; ++q) sm[q][threadIdx.x] = s[q];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      for (int q = 0; q < 5; ++q) sm[q][threadIdx.x] += sm[q][threadIdx.x + w];
      sm[5][threadIdx.x] = fmax(sm[5][threadIdx.x], sm[5][threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < 6; ++q) out[q] = sm[q][0];
}

template <typename R>
static aeth_status diag_T(aeth_ctx* c) {
  const int nb = (int)c->blocks.size();
  k_diag<R><<<c->dt_grid, 256, 0, c->stream>>>((const BlockPtrs<R>*)c->d_tab,
                                               c->d_prefix + PK_ROWS * (nb + 1), nb,
                                               prefix_total(c, PK_ROWS), is_mhd(c), c->d_partials);
  k_diag_final<<<1, 256, 0, c->stream>>>(c->d_partials, c->dt_grid, c->d_diag);
  AETH_CK(c, cudaGetLastError());
  return AETH_OK;
}

aeth_status enqueue_diag(aeth_ctx* c) {
  return c->elem == 8 ? diag_T<double>(c) : diag_T<float>(c);
}

}  // namespace aeth
