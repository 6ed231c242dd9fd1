// C ABI of the SACRA-2D hot path (include/sacra2d.h): contexts, device arena,
// the stage sequence of Sec. II.D (lockstep levels), batched persistent
// launches over all levels of one star or of many stars, the autotuner of
// their tile shapes and grid sizes, and CUDA-graph replay of whole steps.  All
// arithmetic runs in the kernels of hydro.cu, z4c.cu and grid.cu; the host
// orders launches, builds tile lists and computes interpolation weights.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "kernels.h"

using namespace sacra;

namespace {

constexpr int kMaxLevels = 12;
constexpr int kTabStride = 12;   // 9 weights, cos, sin, cos - 1

// Lagrange weights over the nodes at position t (product formula)
void lagrange_weights(int n, const double *nodes, double t, double *w) {
  for (int a = 0; a < n; ++a) {
    double v = 1.0;
    for (int b = 0; b < n; ++b)
      if (b != a) v *= (t - nodes[b]) / (nodes[a] - nodes[b]);
    w[a] = v;
  }
}

size_t round_up(size_t v, size_t m) { return (v + m - 1) / m * m; }

// levels [0, G) share the coarse step; levels >= G take half their parent's step
int lockstep_levels(const sacra_params *p) {
  const int K = p->subcycle_from;
  return (K <= 0 || K >= p->n_levels) ? p->n_levels : K;
}

// time slices a parent of a sub-cycled level keeps (Sec. II.D): the metric at
// t^{n-1} and the interpolant, the primitives at t^{n-1}, t^n and the interpolant
constexpr int kSubPlanes = 2 * NMET + 3 * NPRIM;

// Device memory of one star (hierarchy): per level the state registers,
// primitives, face fluxes, its own derivative and cartoon scratch (the levels
// of a stage run concurrently), the time slices when sub-cycling, flux
// registers and status; then the diagnostic partial sums.
struct Layout {
  size_t P;          // plane stride (doubles), multiple of 32
  int rw;            // flux register row width
  size_t per_level;  // bytes
  size_t part_bytes; // diagnostic partials
  int n_part;
};

Layout layout(const sacra_params *p) {
  Layout o;
  const size_t px = p->nx + 2 * GH, pz = p->nz + 2 * GH;
  o.P = round_up(px * pz, 32);
  o.rw = (p->nx > p->nz ? p->nx : p->nz) + 2;
  const size_t rwp = round_up((size_t)o.rw, 32);
  const size_t planes = 4 * NST + NPRIM + 2 * NCONS + (size_t)z4c_scratch_planes() + 2 * NMET +
                        (lockstep_levels(p) < p->n_levels ? kSubPlanes : 0);
  o.per_level = round_up(planes * o.P * 8 + o.P * 4 /* status */ + 4 * NCONS * rwp * 8, 256);
  o.n_part = p->n_levels * ((p->nx * p->nz + 127) / 128);
  o.part_bytes = round_up((size_t)o.n_part * 9 * 8, 256);
  return o;
}

size_t star_bytes(const sacra_params *p) {
  const Layout o = layout(p);
  return o.per_level * p->n_levels + o.part_bytes + round_up(sizeof(PwpTable), 256);
}

bool valid(const sacra_params *p, std::string *why) {
  if (!p) { *why = "params is NULL"; return false; }
  if (p->n_levels < 1 || p->n_levels > kMaxLevels) { *why = "n_levels must be in [1, 12]"; return false; }
  if (p->nx < 8 || p->nz < 4) { *why = "nx >= 8 and nz >= 4 required"; return false; }
  if (p->geometry != SACRA_PLANAR && p->geometry != SACRA_CYLINDRICAL) { *why = "unknown geometry"; return false; }
  if (p->n_levels > 1 && (p->nx != p->nz || p->nx % 2 || p->nx < 16 || p->geometry != SACRA_CYLINDRICAL)) {
    *why = "FMR needs nx == nz, even, >= 16, cylindrical geometry";
    return false;
  }
  if (p->geometry == SACRA_PLANAR && p->evolve_spacetime) { *why = "spacetime evolution needs the cylindrical (cartoon) geometry"; return false; }
  if (p->rk != SACRA_RK4 && p->rk != SACRA_SSPRK3) { *why = "unknown integrator"; return false; }
  if (p->solver != SACRA_HLLC && p->solver != SACRA_TVDLF) { *why = "unknown Riemann solver"; return false; }
  if (!(p->dx0 > 0) || !(p->dz0 > 0)) { *why = "dx0, dz0 must be positive"; return false; }
  if (p->evolve_spacetime && fabs(p->dx0 - p->dz0) > 1e-12 * p->dx0) { *why = "cartoon needs dx0 == dz0"; return false; }
  if (!(p->Gamma_th > 1.0) || (p->K != 0.0 && !(p->Gamma > 1.0))) { *why = "EOS indices must exceed 1"; return false; }
  if (!(p->rho_atm > 0) || !(p->w_max > 1) || !(p->c2p_tol > 0) || p->c2p_maxit < 1) { *why = "bad recovery parameters"; return false; }
  if (p->precision & ~SACRA_MIXED) { *why = "unknown precision bits"; return false; }
  if (p->subcycle_from < 0) { *why = "subcycle_from must be >= 0"; return false; }
  if (p->hydro_outer != 0 && p->hydro_outer != 1) { *why = "hydro_outer must be 0 or 1"; return false; }
  if (!(p->r_hold >= 0.0)) { *why = "r_hold must be >= 0"; return false; }
  if (p->eos_adiabatic != 0 && p->eos_adiabatic != 1) { *why = "eos_adiabatic must be 0 or 1"; return false; }
  if (p->bssn != 0 && p->bssn != 1) { *why = "bssn must be 0 or 1"; return false; }
  if (p->eos_adiabatic && !(p->K > 0.0)) { *why = "the adiabatic EOS needs a cold part (K > 0)"; return false; }
  if (p->n_pieces < 0 || p->n_pieces > kMaxPieces) { *why = "n_pieces must be in [0, 8]"; return false; }
  if (p->n_pieces > 1) {
    if (!(p->K > 0.0)) { *why = "piecewise polytropes need K > 0"; return false; }
    for (int i = 0; i + 1 < p->n_pieces; ++i) {
      if (!(p->pwp_rho[i] > (i ? p->pwp_rho[i - 1] : 0.0))) { *why = "pwp_rho must increase from > 0"; return false; }
      if (!(p->pwp_Gamma[i] > 1.0)) { *why = "pwp_Gamma must exceed 1"; return false; }
    }
  }
  return true;
}

// stars of one batch share the choices that select kernels (geometry, spacetime
// evolution, Riemann solver, integrator, precision); every other parameter
// (grid, EOS, gauge, atmosphere, recovery) is the star's own
bool compatible(const sacra_params *a, const sacra_params *b) {
  return a->geometry == b->geometry && a->evolve_spacetime == b->evolve_spacetime && a->solver == b->solver &&
         a->rk == b->rk && a->precision == b->precision;
}

// kernel kinds for launch counting and the optional per-kernel profile
enum Kid {
  K_OUTFLOW, K_OUTER, K_PROLONG, K_PARITY_X, K_PARITY_Z, K_FLUX_X, K_FLUX_Z, K_HYDRO_DIV, K_CARTOON, K_Z4C_DERIVS,
  K_Z4C_POINT, K_RK_UPDATE, K_RESTRICT, K_REFLUX, K_C2P, K_PRIM2CONS, K_DIAG, K_DIAG_FINAL, K_TIME_INTERP, K_COUNT
};
const char *kKidName[K_COUNT] = {"k_outflow", "k_outer", "k_prolong", "k_parity_x", "k_parity_z", "k_flux_x",
                                 "k_flux_z", "k_hydro_rhs", "k_cartoon", "k_z4c_derivs", "k_z4c_point",
                                 "k_rk_update", "k_restrict", "k_reflux", "k_c2p_region", "k_prim2cons_all",
                                 "k_diag", "k_diag_final", "k_time_interp"};
const Kid kKindKid[B_NKIND] = {K_FLUX_X, K_FLUX_Z, K_HYDRO_DIV, K_CARTOON, K_Z4C_DERIVS, K_Z4C_POINT, K_RK_UPDATE};

struct ProfRec {
  int kid;
  cudaEvent_t a, b;
  long long cells;
};

// one hierarchy of levels
struct Star {
  sacra_params prm;
  DevParams dp;
  Layout lay;
  Lev lv[kMaxLevels];
  void *ds[kMaxLevels];
  double *part = nullptr;
  double dt_step = 0.0;
  bool have_data[kMaxLevels] = {};
  int G = 1;                      // levels [0, G) share the coarse step
  int lpar[kMaxLevels] = {};      // register swaps of each level mod 2
  // time slices of a parent of a sub-cycled level (levels >= G - 1 with a child)
  double *uold[kMaxLevels] = {}, *pold[kMaxLevels] = {}, *pnow[kMaxLevels] = {};
  double *ut[kMaxLevels] = {}, *pt[kMaxLevels] = {};
  bool have_old[kMaxLevels] = {};
  PwpTable *pwp = nullptr;        // device copy of the cold pieces
};

// launch group of level l: 0 = the lockstep levels, then one per sub-cycled level
int group_of(const Star &st, int l) { return l < st.G ? 0 : l - st.G + 1; }

// ---- tile shapes and the autotuner's choice per kernel kind
struct Shape {
  int x, y;
};
const Shape kShapes128[] = {{32, 4}, {64, 2}, {16, 8}, {128, 1}};
const Shape kShapes256[] = {{32, 4}, {64, 2}, {16, 8}, {128, 1}, {32, 8}, {64, 4}};
const int kBlocksPerSm[] = {1, 2, 3, 4, 6, 8, 12};

// the launch bounds (threads per block) of the batched kernels
int max_threads(int kind) {
  switch (kind) {
    case B_FLUX_X: case B_FLUX_Z: case B_HYDRO: case B_DERIVS: return 256;
    default: return 128;
  }
}

struct KindCfg {
  Shape shape{32, 4};
  int blocks_per_sm = 8;
};

struct Region {
  int j0, j1, k0, k1;
};

// cells a kind covers on level l of a star at stage s
Region kind_region(const sacra_params &p, int l, int s, int S, int kind) {
  const int ext = (l > 0 && s < S - 1) ? 4 : 0;
  const int jmax = p.nx + ext, kmax = p.nz + ext;
  switch (kind) {
    case B_FLUX_X: return {0, jmax, 1, kmax};
    case B_FLUX_Z: return {1, jmax, 0, kmax};
    case B_CARTOON: return {-2, p.nx + 4, -2, p.nz + 7};
    default: return {1, jmax, 1, kmax};
  }
}

long long tile_count(const Region &r, Shape sh) {
  return (long long)((r.j1 - r.j0 + sh.x) / sh.x) * ((r.k1 - r.k0 + sh.y) / sh.y);
}

}  // namespace

// The execution engine behind both public handles: one star (sacra_ctx) or a
// batch of stars advanced together (sacra_batch).
struct Engine {
  std::vector<Star> stars;
  DevParams dp;
  int S = 4;                      // stages per step
  cudaStream_t stream = nullptr;
  // uploads of a level's state (set_initial_data, RAW): the host-to-device
  // copy runs in row chunks on its own stream, each chunk's recovery on the
  // context's stream as soon as that chunk has arrived
  static constexpr int kUpChunks = 8;
  cudaStream_t up_stream = nullptr;
  cudaEvent_t up_start = nullptr, up_chunk[kUpChunks] = {};
  char *arena = nullptr;
  bool own_arena = false;
  double *tab = nullptr, *tabw = nullptr, *dout = nullptr;
  unsigned long long *nfb = nullptr;
  int *tctr = nullptr;            // the tile counter of the batched launches (zeroed before each)
  int sms = 1;
  // plan of the batched launches
  std::vector<std::pair<int, int>> slots;   // (star, level)
  std::vector<int> slot_group;    // launch group of each slot
  std::vector<int> group_first;   // first slot of each group
  int ngroups = 1;
  BL *bl_dev = nullptr;           // [2 parities][S][slots], then 2 x slots tuning copies
  Tile *tiles_dev = nullptr;
  size_t tiles_cap = 0, tune_cap = 0;
  std::vector<long long> toff, tcnt, cells;   // [group][stage][kind]
  KindCfg cfg[B_NKIND];
  // level lists of the lockstep step (kernels.h, LItem): the ghost fill and the
  // restriction as one launch per operation and level depth over every star
  struct LList {
    long long off = 0;       // first item in litems_dev
    int n = 0, max_nx = 0;   // items, the largest nx among them
    long long cells = 0;     // units of work (profiling)
  };
  LItem *litems_dev = nullptr;
  size_t litems_cap = 0;
  int lmax = 0;                        // the largest level count of the stars
  bool lists = false;                  // the lockstep step runs on the level lists
  std::vector<LList> l_fill, l_fpar;   // [parity][stage][depth]: outer (depth 0) / prolongation; parity
  std::vector<LList> l_restr, l_rpar;  // [parity][depth]: restriction of depth onto depth - 1; child parity
  LList l_oend[2], l_ppar[2];          // [parity]: outer boundary after the last stage; parents' parity
  // bookkeeping
  long long launches = 0;
  std::string err;
  // step graphs, keyed by 2 * parity + (diagnostics in the first stage)
  cudaGraphExec_t gexec[4] = {nullptr, nullptr, nullptr, nullptr};
  double gdt[4] = {0.0, 0.0, 0.0, 0.0};
  long long glaunch[4] = {0, 0, 0, 0};
  bool stage0_diag = false;       // enqueue the diagnostics inside the first stage of each step
  int parity = 0;    // register swaps of group 0 mod 2 (the key of the step graphs)
  bool capturing = false;
  bool prof = false;
  std::vector<ProfRec> recs;
  std::vector<cudaEvent_t> pool;
  size_t pool_used = 0;
};

struct sacra_ctx {
  Engine e;
};
struct sacra_batch {
  Engine e;
};

namespace {

sacra_status fail(Engine &e, sacra_status s, const std::string &m) {
  e.err = m;
  return s;
}

sacra_status cuda_check(Engine &e, const char *where) {
  cudaError_t x = cudaGetLastError();
  if (x != cudaSuccess) return fail(e, SACRA_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(x));
  return SACRA_OK;
}

cudaEvent_t pool_event(Engine &e) {
  if (e.pool_used == e.pool.size()) {
    cudaEvent_t x;
    cudaEventCreate(&x);
    e.pool.push_back(x);
  }
  return e.pool[e.pool_used++];
}

// every kernel launch goes through here: count it, and bracket it with
// events when profiling (not while a graph is being captured)
template <class F>
void run(Engine &e, Kid k, long long cells, F &&launch) {
  if (e.prof && !e.capturing) {
    ProfRec r{(int)k, pool_event(e), pool_event(e), cells};
    cudaEventRecord(r.a, e.stream);
    launch();
    cudaEventRecord(r.b, e.stream);
    e.recs.push_back(r);
  } else {
    launch();
  }
  ++e.launches;
}

double stage_c(int rk, int s) {
  static const double c4[4] = {0.0, 0.5, 0.5, 1.0}, c3[3] = {0.0, 1.0, 0.5};
  return rk == SACRA_RK4 ? c4[s] : c3[s];
}
double stage_b(int rk, int s) {
  static const double b4[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0}, b3[3] = {1.0 / 6.0, 1.0 / 6.0, 2.0 / 3.0};
  return rk == SACRA_RK4 ? b4[s] : b3[s];
}
double *stage_state(Star &st, int l, int s) { return s == 0 ? st.lv[l].un : st.lv[l].us; }

bool kind_used(const Engine &e, int kind) {
  const sacra_params &p = e.stars[0].prm;
  if (kind == B_CARTOON) return p.evolve_spacetime && p.geometry == SACRA_CYLINDRICAL;
  if (kind == B_DERIVS || kind == B_POINT) return p.evolve_spacetime != 0;
  return true;
}

bool fixed_shape(const Engine &, int kind) { return kind == B_DERIVS; }

Shape kind_shape(const Engine &e, int kind) {
  if (fixed_shape(e, kind)) {
    const dim3 b = (e.dp.mixed & SACRA_MIXED_Z4C) ? z4c_derivs_f32_block() : z4c_derivs_f64_block();
    return {(int)b.x, (int)b.y};
  }
  return e.cfg[kind].shape;
}

// ---------------------------------------------------------------- plan

// level views as stage s at register parity par sees them
BL make_bl(const Engine &e, int slot, int par, int s) {
  const Star &st = e.stars[e.slots[slot].first];
  const int l = e.slots[slot].second;
  BL b;
  b.L = st.lv[l];
  b.P = st.dp;
  if (par != st.lpar[l]) std::swap(b.L.un, b.L.us);   // st.lv holds the registers of the current parity
  b.U = s == 0 ? b.L.un : b.L.us;
  b.DS = st.ds[l];
  const int ext = (l > 0 && s < e.S - 1) ? 4 : 0;
  b.jmax = st.prm.nx + ext;
  b.kmax = st.prm.nz + ext;
  b.has_child = l < st.prm.n_levels - 1;
  b.has_parent = l > 0;
  b.wb = stage_b(st.prm.rk, s);
  b.wbp = l >= st.G ? 0.5 * b.wb : b.wb;             // a sub-cycled level registers two steps of dt / 2
  return b;
}

size_t plan_index(int g, int s, int kind) { return ((size_t)g * 4 + s) * B_NKIND + kind; }

// register parity of launch group g (all its levels swap together)
int group_parity(const Engine &e, int g) {
  const auto &sl = e.slots[e.group_first[g]];
  return e.stars[sl.first].lpar[sl.second];
}

// tiles of the slots of group g (every slot for g < 0)
void build_tiles(const Engine &e, int g, int s, int kind, Shape sh, std::vector<Tile> &out) {
  out.clear();
  for (int i = 0; i < (int)e.slots.size(); ++i) {
    if (g >= 0 && e.slot_group[i] != g) continue;
    const Region r = kind_region(e.stars[e.slots[i].first].prm, e.slots[i].second, s, e.S, kind);
    for (int k0 = r.k0; k0 <= r.k1; k0 += sh.y)
      for (int j0 = r.j0; j0 <= r.j1; j0 += sh.x) out.push_back(Tile{i, j0, k0, 0});
  }
}

long long region_cells(const Engine &e, int g, int s, int kind) {
  long long n = 0;
  for (int i = 0; i < (int)e.slots.size(); ++i) {
    if (e.slot_group[i] != g) continue;
    const auto &sl = e.slots[i];
    const Region r = kind_region(e.stars[sl.first].prm, sl.second, s, e.S, kind);
    n += (long long)(r.j1 - r.j0 + 1) * (r.k1 - r.k0 + 1);
  }
  return n;
}

// tiles of (stage s, kind) over all stars at shape sh
long long count_tiles(const std::vector<sacra_params> &ps, int S, int s, int kind, Shape sh) {
  long long n = 0;
  for (const sacra_params &p : ps)
    for (int l = 0; l < p.n_levels; ++l) n += tile_count(kind_region(p, l, s, S, kind), sh);
  return n;
}

// the largest tile count of (stage s, kind) over every shape a launch may use
long long max_tiles(const std::vector<sacra_params> &ps, int S, int s, int kind) {
  long long m = 0;
  for (const Shape &sh : kShapes256) m = std::max(m, count_tiles(ps, S, s, kind, sh));
  const dim3 f = z4c_derivs_f32_block();
  return std::max(m, count_tiles(ps, S, s, kind, Shape{(int)f.x, (int)f.y}));
}

// tile capacity: every stage and kind at its largest count (the groups
// partition the slots, so their lists add up to the same), then a tuning area
void plan_caps(const std::vector<sacra_params> &ps, size_t *cap, size_t *tune) {
  const int S = ps[0].rk == SACRA_RK4 ? 4 : 3;
  *cap = 0;
  *tune = 0;
  for (int s = 0; s < S; ++s)
    for (int kind = 0; kind < B_NKIND; ++kind) {
      const long long m = max_tiles(ps, S, s, kind);
      *cap += (size_t)m;
      if (s == 0) *tune = std::max(*tune, (size_t)m);
    }
}

size_t plan_bytes(const std::vector<sacra_params> &ps) {
  const int S = ps[0].rk == SACRA_RK4 ? 4 : 3;
  size_t nl = 0;
  for (const sacra_params &p : ps) nl += p.n_levels;
  size_t cap, tune;
  plan_caps(ps, &cap, &tune);
  return round_up((2 * (size_t)S + 2) * nl * sizeof(BL), 256) + round_up((cap + tune) * sizeof(Tile), 256);
}

// level l of star st as parity par sees it (st.lv holds the current registers)
Lev level_view(const Star &st, int l, int par) {
  Lev L = st.lv[l];
  if (par != st.lpar[l]) std::swap(L.un, L.us);
  return L;
}

// items of the level lists (counted by litem_count); each list contiguous
void build_lists(Engine &e, std::vector<LItem> &items) {
  items.clear();
  e.lmax = 0;
  bool same = true;
  const sacra_params &p0 = e.stars[0].prm;
  for (const Star &st : e.stars) {
    e.lmax = std::max(e.lmax, st.prm.n_levels);
    same = same && st.prm.geometry == SACRA_CYLINDRICAL && st.prm.evolve_spacetime == p0.evolve_spacetime &&
           st.prm.hydro_outer == p0.hydro_outer && st.prm.rk == p0.rk;
  }
  e.lists = e.ngroups == 1 && same;
  const int D = e.lmax;
  e.l_fill.assign((size_t)2 * e.S * D, Engine::LList());
  e.l_fpar.assign((size_t)2 * e.S * D, Engine::LList());
  e.l_restr.assign((size_t)2 * D, Engine::LList());
  e.l_rpar.assign((size_t)2 * D, Engine::LList());
  auto open = [&](Engine::LList &ll) { ll = Engine::LList(); ll.off = (long long)items.size(); };
  // max_nx: the largest extent in x or z (the launches are sized for it)
  auto add = [&](Engine::LList &ll, const LItem &it, int nx, long long cells) {
    items.push_back(it);
    ++ll.n;
    ll.max_nx = std::max(ll.max_nx, std::max(nx, it.L.nz));
    ll.cells += cells;
  };
  for (int par = 0; par < 2; ++par) {
    for (int s = 0; s < e.S; ++s)
      for (int d = 0; d < D; ++d) {
        Engine::LList &F = e.l_fill[((size_t)par * e.S + s) * D + d];
        open(F);
        for (const Star &st : e.stars) {
          if (st.prm.n_levels <= d) continue;
          LItem it;
          memset(&it, 0, sizeof(it));
          it.L = level_view(st, d, par);
          it.P = st.dp;
          it.B = s == 0 ? it.L.un : it.L.us;
          if (d == 0) {
            it.A = it.L.un;
            add(F, it, st.prm.nx, (long long)(it.L.nx + GH) * (it.L.nz + GH) - (long long)it.L.nx * it.L.nz);
          } else {
            it.Pa = level_view(st, d - 1, par);
            it.A = s == 0 ? it.Pa.un : it.Pa.us;
            add(F, it, st.prm.nx, prolong_cells(it.L, s == 0));
          }
        }
        Engine::LList &Q = e.l_fpar[((size_t)par * e.S + s) * D + d];
        open(Q);
        for (const Star &st : e.stars) {
          if (st.prm.n_levels <= d) continue;
          LItem it;
          memset(&it, 0, sizeof(it));
          it.L = level_view(st, d, par);
          it.P = st.dp;
          it.B = s == 0 ? it.L.un : it.L.us;
          add(Q, it, st.prm.nx, 8LL * (it.L.nz + GH));
        }
      }
    open(e.l_oend[par]);
    for (const Star &st : e.stars) {
      LItem it;
      memset(&it, 0, sizeof(it));
      it.L = level_view(st, 0, par);
      it.P = st.dp;
      it.A = it.L.un;
      it.B = it.L.us;
      add(e.l_oend[par], it, st.prm.nx, (long long)(it.L.nx + GH) * (it.L.nz + GH) - (long long)it.L.nx * it.L.nz);
    }
    for (int d = 1; d < D; ++d) {
      Engine::LList &Q = e.l_rpar[(size_t)par * D + d];
      open(Q);
      for (const Star &st : e.stars) {
        if (st.prm.n_levels <= d) continue;
        LItem it;
        memset(&it, 0, sizeof(it));
        it.L = level_view(st, d, par);
        it.P = st.dp;
        it.B = it.L.un;
        add(Q, it, st.prm.nx, 8LL * (it.L.nz + GH));
      }
      Engine::LList &R = e.l_restr[(size_t)par * D + d];
      open(R);
      for (const Star &st : e.stars) {
        if (st.prm.n_levels <= d) continue;
        LItem it;
        memset(&it, 0, sizeof(it));
        it.L = level_view(st, d, par);
        it.Pa = level_view(st, d - 1, par);
        it.P = st.dp;
        add(R, it, st.prm.nx, (long long)(st.prm.nx / 2) * (st.prm.nx / 2));
      }
    }
    open(e.l_ppar[par]);
    for (const Star &st : e.stars)
      for (int l = 0; l < st.prm.n_levels - 1; ++l) {
        LItem it;
        memset(&it, 0, sizeof(it));
        it.L = level_view(st, l, par);
        it.P = st.dp;
        it.B = it.L.un;
        add(e.l_ppar[par], it, st.prm.nx, 8LL * (it.L.nz + GH));
      }
  }
}

// upload the level views, the tile lists of the current choice of shapes and
// the level lists
sacra_status upload_plan(Engine &e) {
  const int NL = (int)e.slots.size();
  std::vector<LItem> litems;
  build_lists(e, litems);
  if (litems.size() > e.litems_cap) return fail(e, SACRA_ERR_OOM, "level-list capacity exceeded");
  if (!litems.empty())
    cudaMemcpyAsync(e.litems_dev, litems.data(), litems.size() * sizeof(LItem), cudaMemcpyHostToDevice, e.stream);
  std::vector<BL> bls((size_t)2 * e.S * NL);
  for (int par = 0; par < 2; ++par)
    for (int s = 0; s < e.S; ++s)
      for (int i = 0; i < NL; ++i) bls[((size_t)par * e.S + s) * NL + i] = make_bl(e, i, par, s);
  cudaMemcpyAsync(e.bl_dev, bls.data(), bls.size() * sizeof(BL), cudaMemcpyHostToDevice, e.stream);
  std::vector<Tile> all, t;
  const size_t np = plan_index(e.ngroups, 0, 0);
  e.toff.assign(np, 0);
  e.tcnt.assign(np, 0);
  e.cells.assign(np, 0);
  for (int g = 0; g < e.ngroups; ++g)
    for (int s = 0; s < e.S; ++s)
      for (int kind = 0; kind < B_NKIND; ++kind) {
        build_tiles(e, g, s, kind, kind_shape(e, kind), t);
        const size_t i = plan_index(g, s, kind);
        e.toff[i] = (long long)all.size();
        e.tcnt[i] = (long long)t.size();
        e.cells[i] = region_cells(e, g, s, kind);
        all.insert(all.end(), t.begin(), t.end());
      }
  if (all.size() > e.tiles_cap) return fail(e, SACRA_ERR_OOM, "tile capacity exceeded");
  cudaMemcpyAsync(e.tiles_dev, all.data(), all.size() * sizeof(Tile), cudaMemcpyHostToDevice, e.stream);
  // the host vectors must live until the copies are done
  if (cudaStreamSynchronize(e.stream) != cudaSuccess) return cuda_check(e, "upload plan");
  return cuda_check(e, "upload plan");
}

Batch batch_of(const Engine &e, int g, int s, int kind) {
  Batch b;
  b.bl = e.bl_dev + ((size_t)group_parity(e, g) * e.S + s) * e.slots.size();
  b.tiles = e.tiles_dev + e.toff[plan_index(g, s, kind)];
  b.ntiles = (int)e.tcnt[plan_index(g, s, kind)];
  const Shape sh = kind_shape(e, kind);
  b.block = dim3(sh.x, sh.y);
  const long long nb = (long long)e.sms * e.cfg[kind].blocks_per_sm;
  b.grid = (int)std::max(1LL, std::min<long long>(nb, b.ntiles));
  b.ctr = e.tctr;
  return b;
}

void launch_kind(Engine &e, int kind, const Batch &b, int s, double dt) {
  cudaMemsetAsync(b.ctr, 0, sizeof(int), e.stream);   // launches on the one stream: one counter serves all
  switch (kind) {
    case B_FLUX_X: launch_b_flux_x(b, e.dp, e.stream); break;
    case B_FLUX_Z: launch_b_flux_z(b, e.dp, e.stream); break;
    case B_HYDRO: launch_b_hydro_div(b, e.dp, e.stream); break;
    case B_CARTOON: launch_b_cartoon(b, e.dp, e.tab, kTabStride, e.tabw, e.stream); break;
    case B_DERIVS: launch_b_z4c_derivs(b, e.dp, e.stream); break;
    case B_POINT: launch_b_z4c_point(b, e.dp, e.stream, s == 0 && e.stage0_diag ? 1 : 0); break;
    case B_RK: launch_b_rk_update(b, e.dp, s, dt, e.stream); break;
  }
}

// ---------------------------------------------------------------- stage sequence

void enqueue_parity(Engine &e, Star &st, int l, double *U) {
  const Lev &L = st.lv[l];
  run(e, K_PARITY_X, 8LL * (L.nz + GH), [&] { launch_parity_x(L, U, e.stream); });
  run(e, K_PARITY_Z, 8LL * (L.nx + 2 * GH), [&] { launch_parity_z(L, U, e.stream); });
}

void enqueue_fill(Engine &e, Star &st, int s, double dt) {
  for (int l = 0; l < st.prm.n_levels; ++l) {
    double *U = stage_state(st, l, s);
    const Lev &L = st.lv[l];
    if (st.prm.geometry == SACRA_PLANAR) {
      run(e, K_OUTFLOW, (long long)L.px * L.pz, [&] { launch_outflow(L, U, e.stream); });
      continue;
    }
    if (l == 0) {
      run(e, K_OUTER, (long long)(L.nx + GH) * (L.nz + GH) - (long long)L.nx * L.nz,
          [&] { launch_outer(L, st.dp, L.un, U, stage_c(st.prm.rk, s) * dt, e.stream); });
    } else {
      double *Up = stage_state(st, l - 1, s);
      run(e, K_PROLONG, prolong_cells(L, s == 0), [&] { launch_prolong(L, st.lv[l - 1], st.dp, U, Up, s == 0, e.stream); });
      ++e.launches;   // the prolongation is two kernels
    }
    enqueue_parity(e, st, l, U);
  }
}

// ---- the lockstep step on the level lists: one launch per operation and
// level depth over every star (the order within a star is that of
// enqueue_fill / enqueue_restrict: a level's ghost fill reads its parent's
// filled ghosts, a restriction reads its child's restricted interior)

void enqueue_parity_list(Engine &e, const Engine::LList &Q) {
  if (Q.n <= 0) return;
  const LItem *it = e.litems_dev + Q.off;
  run(e, K_PARITY_X, Q.cells, [&] { launch_l_parity_x(it, Q.n, Q.max_nx, e.stream); });
  run(e, K_PARITY_Z, Q.cells, [&] { launch_l_parity_z(it, Q.n, Q.max_nx, e.stream); });
}

void enqueue_fill_lists(Engine &e, int s, double dt) {
  const sacra_params &p0 = e.stars[0].prm;
  const size_t base = ((size_t)e.parity * e.S + s) * e.lmax;
  for (int d = 0; d < e.lmax; ++d) {
    const Engine::LList &F = e.l_fill[base + d];
    const LItem *it = e.litems_dev + F.off;
    if (F.n > 0) {
      if (d == 0) {
        run(e, K_OUTER, F.cells, [&] {
          launch_l_outer(it, F.n, F.max_nx, stage_c(p0.rk, s) * dt, p0.evolve_spacetime, !p0.hydro_outer, e.stream);
        });
      } else {
        run(e, K_PROLONG, F.cells, [&] { launch_l_prolong(it, F.n, F.max_nx, s == 0, e.stream); });
        ++e.launches;   // the prolongation is two kernels
      }
    }
    enqueue_parity_list(e, e.l_fpar[base + d]);
  }
}

void enqueue_restrict_lists(Engine &e, double dt) {
  const size_t base = (size_t)e.parity * e.lmax;
  for (int d = e.lmax - 1; d >= 1; --d) {
    enqueue_parity_list(e, e.l_rpar[base + d]);
    const Engine::LList &R = e.l_restr[base + d];
    if (R.n <= 0) continue;
    const LItem *it = e.litems_dev + R.off;
    run(e, K_RESTRICT, R.cells, [&] { launch_l_restrict(it, R.n, R.max_nx, e.stream); });
    ++e.launches;   // the restriction is two kernels
    run(e, K_REFLUX, (long long)R.n * R.max_nx, [&] { launch_l_reflux(it, R.n, R.max_nx, dt, e.stream); });
    // the restricted cells [1, N/2]^2 and the refluxed strips next to them (not the corner)
    run(e, K_C2P, R.cells, [&] { launch_l_c2p_restricted(it, R.n, R.max_nx, e.stream); });
  }
  // the parents' axis/equator ghosts mirror their restricted interiors
  enqueue_parity_list(e, e.l_ppar[e.parity]);
}

// swap the step and stage registers of the levels of group g
void swap_group(Engine &e, int g) {
  for (size_t i = 0; i < e.slots.size(); ++i) {
    if (e.slot_group[i] != g) continue;
    Star &st = e.stars[e.slots[i].first];
    const int l = e.slots[i].second;
    std::swap(st.lv[l].un, st.lv[l].us);
    st.lpar[l] ^= 1;
  }
  if (g == 0) e.parity ^= 1;
}

// One RK stage of the levels of group g with step dt: one batched launch per
// kernel kind.  At stage 0 the flux registers at each level's child boundary
// are cleared, those at its parent boundary when reset_parent is set (a
// sub-cycled level sums them over both of its steps inside a parent step).
// After the last stage: level 0's outer boundary, then the register swap.
void enqueue_diag(Engine &e, Star &st, bool own_derivs);

void enqueue_group_stage(Engine &e, int g, int s, double dt, bool reset_parent) {
  if (s == 0)
    for (size_t i = 0; i < e.slots.size(); ++i) {
      if (e.slot_group[i] != g) continue;
      Star &st = e.stars[e.slots[i].first];
      const Lev &L = st.lv[e.slots[i].second];
      const size_t reg = (size_t)NCONS * L.rw;   // doubles per register
      if (g == 0) st.dt_step = dt;
      if (reset_parent) {
        cudaMemsetAsync(L.freg, 0, 4 * reg * sizeof(double), e.stream);
      } else {
        cudaMemsetAsync(L.freg, 0, reg * sizeof(double), e.stream);
        cudaMemsetAsync(L.freg + 2 * reg, 0, reg * sizeof(double), e.stream);
      }
    }
  // the hydro sources read the first derivatives the derivative pass has
  // formed, so they follow it
  static const int kOrder[B_NKIND] = {B_FLUX_X, B_FLUX_Z, B_CARTOON, B_DERIVS, B_HYDRO, B_POINT, B_RK};
  for (int ko = 0; ko < B_NKIND; ++ko) {
    const int kind = kOrder[ko];
    // the diagnostics of the state at the start of the step read the
    // derivative scratch and the Ricci scalar the stage has just formed,
    // before the stage update overwrites the primitives
    if (kind == B_RK && s == 0 && g == 0 && e.stage0_diag)
      for (Star &st : e.stars) enqueue_diag(e, st, false);
    if (!kind_used(e, kind)) continue;
    const Batch b = batch_of(e, g, s, kind);
    run(e, kKindKid[kind], e.cells[plan_index(g, s, kind)], [&] { launch_kind(e, kind, b, s, dt); });
  }
  if (s == e.S - 1) {
    if (g == 0 && e.lists) {
      const Engine::LList &O = e.l_oend[e.parity];
      const sacra_params &p0 = e.stars[0].prm;
      run(e, K_OUTER, O.cells, [&] {
        launch_l_outer(e.litems_dev + O.off, O.n, O.max_nx, dt, p0.evolve_spacetime, !p0.hydro_outer, e.stream);
      });
    } else if (g == 0)
      for (Star &st : e.stars)
        if (st.prm.geometry == SACRA_CYLINDRICAL) {
          const Lev &L0 = st.lv[0];
          run(e, K_OUTER, (long long)(L0.nx + GH) * (L0.nz + GH) - (long long)L0.nx * L0.nz,
              [&] { launch_outer(L0, st.dp, L0.un, L0.us, dt, e.stream); });
        }
    swap_group(e, g);
  }
}

// one RK stage of every level of every star (all levels with the same dt)
void enqueue_stage(Engine &e, int s, double dt) {
  for (int g = 0; g < e.ngroups; ++g) enqueue_group_stage(e, g, s, dt, true);
}

void enqueue_restrict(Engine &e, Star &st) {
  const int L = st.prm.n_levels;
  if (L < 2) return;
  for (int l = L - 1; l >= 1; --l) {
    Lev &C = st.lv[l], &Pa = st.lv[l - 1];
    enqueue_parity(e, st, l, C.un);
    const int nh = Pa.nx / 2;
    run(e, K_RESTRICT, (long long)nh * nh, [&] { launch_restrict(C, Pa, e.stream); });
    ++e.launches;   // the restriction is two kernels
    run(e, K_REFLUX, 2LL * nh, [&] { launch_reflux(C, Pa, st.dt_step, e.stream); });
    // the restricted cells [1, N/2]^2 and the refluxed strips next to them (not the corner)
    run(e, K_C2P, (long long)(nh + 1) * (nh + 1) - 1,
        [&] { launch_c2p_region(Pa, st.dp, Pa.un, 1, nh + 1, 1, nh + 1, e.stream, 1); });
  }
  // the parents' axis/equator ghosts mirror their restricted interiors
  for (int l = 0; l < L - 1; ++l) enqueue_parity(e, st, l, st.lv[l].un);
}

// ---- Berger-Oliger sub-cycling (Sec. II.D)

// restriction of level l onto its parent and reflux with the parent's step dt,
// recovery there, and the parent's axis/equator ghosts
void enqueue_restrict_pair(Engine &e, Star &st, int l, double dt) {
  Lev &C = st.lv[l], &Pa = st.lv[l - 1];
  enqueue_parity(e, st, l, C.un);
  const int nh = Pa.nx / 2;
  run(e, K_RESTRICT, (long long)nh * nh, [&] { launch_restrict(C, Pa, e.stream); });
  ++e.launches;   // the restriction is two kernels
  run(e, K_REFLUX, 2LL * nh, [&] { launch_reflux(C, Pa, dt, e.stream); });
  run(e, K_C2P, (long long)(nh + 1) * (nh + 1) - 1,
      [&] { launch_c2p_region(Pa, st.dp, Pa.un, 1, nh + 1, 1, nh + 1, e.stream, 1); });
  enqueue_parity(e, st, l - 1, Pa.un);
}

// the primitives at t^n of a parent, taken at the start of its step
void save_now(Engine &e, Star &st, int l) {
  const Lev &L = st.lv[l];
  cudaMemcpyAsync(st.pnow[l], L.prim, (size_t)NPRIM * L.P * sizeof(double), cudaMemcpyDeviceToDevice, e.stream);
}

// after a parent step and its children's: the t^n slice becomes t^{n-1}
void rotate_slices(Engine &e, Star &st, int l) {
  const Lev &L = st.lv[l];
  cudaMemcpyAsync(st.uold[l], L.us, (size_t)NMET * L.P * sizeof(double), cudaMemcpyDeviceToDevice, e.stream);
  cudaMemcpyAsync(st.pold[l], st.pnow[l], (size_t)NPRIM * L.P * sizeof(double), cudaMemcpyDeviceToDevice, e.stream);
  st.have_old[l] = true;
}

// buffer zone of sub-cycled level l at stage s from its parent at t^n + theta dt_parent
void enqueue_sub_fill(Engine &e, Star &st, int l, int s, double theta) {
  const Lev &L = st.lv[l];
  const Lev &Pa = st.lv[l - 1];
  double *U = stage_state(st, l, s);
  const long long np = (long long)Pa.px * Pa.pz;
  run(e, K_TIME_INTERP, np * (NMET + NPRIM), [&] {
    launch_time_interp(Pa, st.uold[l - 1], st.pold[l - 1], st.pnow[l - 1], st.ut[l - 1], st.pt[l - 1], theta,
                       st.have_old[l - 1] ? 1 : 0, e.stream);
  });
  Lev Pt = Pa;
  Pt.prim = st.pt[l - 1];
  run(e, K_PROLONG, prolong_cells(L, s == 0), [&] { launch_prolong(L, Pt, st.dp, U, st.ut[l - 1], s == 0, e.stream); });
  ++e.launches;   // the prolongation is two kernels
  enqueue_parity(e, st, l, U);
}

// two steps of dtl of sub-cycled level l inside one step of its parent
void advance_sub(Engine &e, Star &st, int l, double dtl) {
  const int L = st.prm.n_levels, g = group_of(st, l);
  for (int m = 0; m < 2; ++m) {
    for (int s = 0; s < e.S; ++s) {
      enqueue_sub_fill(e, st, l, s, 0.5 * (m + stage_c(st.prm.rk, s)));
      if (s == 0 && l + 1 < L) save_now(e, st, l);
      enqueue_group_stage(e, g, s, dtl, m == 0);
    }
    if (l + 1 < L) {
      enqueue_parity(e, st, l, st.lv[l].un);
      advance_sub(e, st, l + 1, 0.5 * dtl);
      enqueue_restrict_pair(e, st, l + 1, dtl);
      rotate_slices(e, st, l);
    }
  }
}

// one coarse step of a sub-cycled star: the lockstep levels [0, G) with dt,
// each deeper level twice per step of its parent, restriction and reflux
// whenever a child has caught up with its parent
void enqueue_step_sub(Engine &e, Star &st, double dt) {
  const int G = st.G;
  for (int s = 0; s < e.S; ++s) {
    for (int l = 0; l < G; ++l) {
      double *U = stage_state(st, l, s);
      const Lev &Lv = st.lv[l];
      if (l == 0) {
        run(e, K_OUTER, (long long)(Lv.nx + GH) * (Lv.nz + GH) - (long long)Lv.nx * Lv.nz,
            [&] { launch_outer(Lv, st.dp, Lv.un, U, stage_c(st.prm.rk, s) * dt, e.stream); });
      } else {
        double *Up = stage_state(st, l - 1, s);
        run(e, K_PROLONG, prolong_cells(Lv, s == 0),
            [&] { launch_prolong(Lv, st.lv[l - 1], st.dp, U, Up, s == 0, e.stream); });
        ++e.launches;
      }
      enqueue_parity(e, st, l, U);
    }
    if (s == 0) save_now(e, st, G - 1);
    enqueue_group_stage(e, 0, s, dt, true);
  }
  enqueue_parity(e, st, G - 1, st.lv[G - 1].un);
  advance_sub(e, st, G, 0.5 * dt);
  enqueue_restrict_pair(e, st, G, dt);
  rotate_slices(e, st, G - 1);
  for (int l = G - 1; l >= 1; --l) enqueue_restrict_pair(e, st, l, dt);
}

void enqueue_step(Engine &e, double dt) {
  if (e.ngroups > 1) {           // a sub-cycled star (single contexts only)
    enqueue_step_sub(e, e.stars[0], dt);
    return;
  }
  if (e.lists) {
    for (int s = 0; s < e.S; ++s) {
      enqueue_fill_lists(e, s, dt);
      enqueue_stage(e, s, dt);
    }
    enqueue_restrict_lists(e, dt);
    return;
  }
  for (int s = 0; s < e.S; ++s) {
    for (Star &st : e.stars) enqueue_fill(e, st, s, dt);
    enqueue_stage(e, s, dt);
  }
  for (Star &st : e.stars) enqueue_restrict(e, st);
}

// every parent of a sub-cycled level holds a t^{n-1} slice (the time
// interpolation's order is then fixed, and a captured step can be replayed)
bool steady(const Engine &e) {
  for (const Star &st : e.stars)
    for (int l = st.G - 1; l < st.prm.n_levels - 1; ++l)
      if (!st.have_old[l]) return false;
  return true;
}

bool ready(const Engine &e) {
  for (const Star &st : e.stars)
    for (int l = 0; l < st.prm.n_levels; ++l)
      if (!st.have_data[l]) return false;
  return true;
}

void drop_graphs(Engine &e) {
  for (int i = 0; i < 4; ++i)
    if (e.gexec[i]) {
      cudaGraphExecDestroy(e.gexec[i]);
      e.gexec[i] = nullptr;
    }
}

// ---------------------------------------------------------------- autotuner
//
// Per kernel kind: every tile shape the kernel's launch bounds allow, times
// every persistent grid size (blocks per SM), each timed by CUDA events over
// `reps` stage-0 launches on the current state.  These launches change no
// state: the flux registers are off, the stage update writes into the level's
// derivative scratch, the fallback counter is restored afterwards, and every
// buffer they do write (face fluxes, right-hand sides, scratch) is recomputed
// by the next stage.
sacra_status tune(Engine &e, int reps) {
  if (!ready(e)) return fail(e, SACRA_ERR_STATE, "initial data missing on some level");
  if (reps < 1) reps = 1;
  drop_graphs(e);
  const int NL = (int)e.slots.size();
  std::vector<BL> tv(2 * (size_t)NL);
  for (int i = 0; i < NL; ++i) {
    BL b = make_bl(e, i, e.stars[e.slots[i].first].lpar[e.slots[i].second], 0);
    b.has_child = b.has_parent = 0;
    tv[i] = b;
    double *scr = reinterpret_cast<double *>(b.DS);
    const size_t P = b.L.P;
    b.L.us = scr;
    b.L.ka = scr + (size_t)NST * P;
    b.L.prim = scr + (size_t)2 * NST * P;
    b.L.status = reinterpret_cast<int *>(scr + (size_t)(2 * NST + NPRIM) * P);
    tv[NL + i] = b;
  }
  BL *tv_dev = e.bl_dev + (size_t)2 * e.S * NL;
  cudaMemcpyAsync(tv_dev, tv.data(), tv.size() * sizeof(BL), cudaMemcpyHostToDevice, e.stream);
  unsigned long long nfb0 = 0;
  cudaMemcpyAsync(&nfb0, e.nfb, sizeof(nfb0), cudaMemcpyDeviceToHost, e.stream);
  if (cudaStreamSynchronize(e.stream) != cudaSuccess) return cuda_check(e, "tune");
  Tile *tune_tiles = e.tiles_dev + e.tiles_cap;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  std::vector<Tile> t;
  sacra_status status = SACRA_OK;
  // coordinate descent per kind: the grid size at the current shape, then the shape at that grid size
  auto time_cfg = [&](int kind, Shape sh, int m, float *ms) -> sacra_status {
    build_tiles(e, -1, 0, kind, sh, t);
    if (t.size() > e.tune_cap) { *ms = 1e30f; return SACRA_OK; }
    cudaMemcpyAsync(tune_tiles, t.data(), t.size() * sizeof(Tile), cudaMemcpyHostToDevice, e.stream);
    Batch bt;
    bt.bl = tv_dev + (kind == B_RK ? NL : 0);
    bt.tiles = tune_tiles;
    bt.ntiles = (int)t.size();
    bt.block = dim3(sh.x, sh.y);
    bt.grid = (int)std::max(1LL, std::min<long long>((long long)e.sms * m, bt.ntiles));
    bt.ctr = e.tctr;
    launch_kind(e, kind, bt, 0, 0.0);   // warm-up
    cudaEventRecord(a, e.stream);
    for (int r = 0; r < reps; ++r) launch_kind(e, kind, bt, 0, 0.0);
    cudaEventRecord(b, e.stream);
    if (cudaEventSynchronize(b) != cudaSuccess) return cuda_check(e, "tune");
    e.launches += reps + 1;
    cudaEventElapsedTime(ms, a, b);
    return SACRA_OK;
  };
  for (int kind = 0; kind < B_NKIND && status == SACRA_OK; ++kind) {
    if (!kind_used(e, kind)) continue;
    std::vector<Shape> shapes;
    if (fixed_shape(e, kind)) shapes.push_back(kind_shape(e, kind));
    else if (max_threads(kind) >= 256) shapes.assign(std::begin(kShapes256), std::end(kShapes256));
    else shapes.assign(std::begin(kShapes128), std::end(kShapes128));
    KindCfg pick = e.cfg[kind];
    pick.shape = kind_shape(e, kind);
    float best = 1e30f;
    for (int m : kBlocksPerSm) {
      float ms = 0.f;
      if ((status = time_cfg(kind, pick.shape, m, &ms)) != SACRA_OK) break;
      if (ms < best) { best = ms; pick.blocks_per_sm = m; }
    }
    for (const Shape &sh : shapes) {
      if (status != SACRA_OK || (sh.x == pick.shape.x && sh.y == pick.shape.y)) continue;
      float ms = 0.f;
      if ((status = time_cfg(kind, sh, pick.blocks_per_sm, &ms)) != SACRA_OK) break;
      if (ms < best) { best = ms; pick.shape = sh; }
    }
    e.cfg[kind] = pick;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (status != SACRA_OK) return status;
  cudaMemcpyAsync(e.nfb, &nfb0, sizeof(nfb0), cudaMemcpyHostToDevice, e.stream);
  status = upload_plan(e);
  if (status != SACRA_OK) return status;
  return cuda_check(e, "tune");
}

// ---------------------------------------------------------------- set-up

void init_star_levels(Star &st, char *base) {
  const sacra_params *p = &st.prm;
  const size_t P = st.lay.P;
  const size_t rwp = round_up((size_t)st.lay.rw, 32);
  for (int l = 0; l < p->n_levels; ++l) {
    Lev &L = st.lv[l];
    memset(&L, 0, sizeof(L));
    char *b = base + st.lay.per_level * l;
    L.nx = p->nx; L.nz = p->nz; L.px = p->nx + 2 * GH; L.pz = p->nz + 2 * GH; L.rw = (int)rwp;
    set_spacing(L, p->dx0 / (double)(1 << l), p->dz0 / (double)(1 << l));
    L.P = P;
    double *dp = (double *)b;
    L.un = dp; dp += NST * P;
    L.us = dp; dp += NST * P;
    L.ka = dp; dp += NST * P;
    L.rhs = dp; dp += NST * P;
    L.rhsq = L.rhs + (size_t)fQD * P;
    L.prim = dp; dp += NPRIM * P;
    L.fx = dp; dp += NCONS * P;
    L.fz = dp; dp += NCONS * P;
    st.ds[l] = dp; dp += (size_t)z4c_scratch_planes() * P;
    L.dy = dp; dp += NMET * P;
    L.dyy = dp; dp += NMET * P;
    if (st.G < p->n_levels) {
      st.uold[l] = dp; dp += NMET * P;
      st.ut[l] = dp; dp += NMET * P;
      st.pold[l] = dp; dp += NPRIM * P;
      st.pnow[l] = dp; dp += NPRIM * P;
      st.pt[l] = dp; dp += NPRIM * P;
    }
    L.freg = dp; dp += 4 * NCONS * rwp;
    L.status = (int *)dp;
  }
  st.part = (double *)(base + st.lay.per_level * p->n_levels);
  st.pwp = (PwpTable *)(base + st.lay.per_level * p->n_levels + st.lay.part_bytes);
}

// shared tables: cartoon weights (for the largest nx) and the grid weights
void upload_tables(Engine &e, int max_nx) {
  // cartoon table: for x_j = (j - 1/2) dx and plane m dy (dy = dx), the 9
  // weights on x_{j-4..j+4} at varpi = sqrt(x_j^2 + (m dy)^2), cos, sin of phi, cos - 1
  const int nj = max_nx + 8;
  std::vector<double> tab((size_t)nj * 3 * kTabStride, 0.0);
  double nodes[9];
  for (int n = 0; n < 9; ++n) nodes[n] = n - 4;
  for (int j = 1; j < nj; ++j)
    for (int m = 1; m <= 3; ++m) {
      const double x = j - 0.5, vp = sqrt(x * x + (double)(m * m));
      double *t = &tab[(size_t)(j * 3 + m - 1) * kTabStride];
      lagrange_weights(9, nodes, vp - x, t);
      t[9] = x / vp;
      t[10] = m / vp;
      t[11] = -(double)(m * m) / (vp * (x + vp));   // cos phi - 1 without cancellation
    }
  // combined weights of the FP64 kernel (kernels.h): with t_m the weights above, c_m = cos,
  // s_m = sin, w1 = (45, -9, 1), w2 = (270, -27, 2):
  //   Sd = sum_m 2 w2 t_m      (d_yy of a scalar, on u_n - u_0)
  //   D1 = -2 sum_m w1 s_m t_m (d_y of v_x from v_y; d_y v_y = -(D1 . v_x))
  //   E1 = -4 sum_m w1 c_m s_m t_m (d_y T_xx from T_xy; d_y T_xy = -E1 . (T_xx - T_yy) / 2)
  //   C2 = sum_m 2 w2 c_m t_m, K2 = sum_m 2 w2 (c_m - 1) (d_yy of a vector component, T_xz, T_yz)
  //   F = sum_m 2 w2 c_m^2 t_m, G = sum_m 2 w2 s_m^2 t_m, H = sum_m 2 w2 (c_m^2 - s_m^2) t_m,
  //   Kb = sum_m 2 w2 s_m^2    (d_yy of T_xx, T_yy, T_xy)
  std::vector<double> tw((size_t)nj * kCartoonW, 0.0);
  const double w1[3] = {45.0, -9.0, 1.0}, w2[3] = {270.0, -27.0, 2.0};
  for (int j = 1; j < nj; ++j) {
    double *W = &tw[(size_t)j * kCartoonW];
    for (int m = 0; m < 3; ++m) {
      const double *t = &tab[(size_t)(j * 3 + m) * kTabStride];
      const double c = t[9], sn = t[10], cm1 = t[11];
      for (int n = 0; n < 9; ++n) {
        W[n] += 2.0 * w2[m] * t[n];
        W[9 + n] += -2.0 * w1[m] * sn * t[n];
        W[18 + n] += -4.0 * w1[m] * c * sn * t[n];
        W[27 + n] += 2.0 * w2[m] * c * t[n];
        W[36 + n] += 2.0 * w2[m] * c * c * t[n];
        W[45 + n] += 2.0 * w2[m] * sn * sn * t[n];
        W[54 + n] += 2.0 * w2[m] * (c * c - sn * sn) * t[n];
      }
      W[63] += 2.0 * w2[m] * cm1;
      W[64] += 2.0 * w2[m] * sn * sn;
    }
  }
  cudaMemcpyAsync(e.tab, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice, e.stream);
  cudaMemcpyAsync(e.tabw, tw.data(), tw.size() * sizeof(double), cudaMemcpyHostToDevice, e.stream);
  GridWeights w;
  double n8[8];
  for (int n = 0; n < 8; ++n) n8[n] = n - 3;
  lagrange_weights(8, n8, 0.25, w.prol);
  lagrange_weights(8, n8, 0.5, w.rest_c);          // nodes 2j-4..2j+3 relative to 2j-1
  for (int n = 0; n < 8; ++n) n8[n] = n;
  lagrange_weights(8, n8, 4.5, w.rest_s1);         // N-7..N -> N - 5/2
  lagrange_weights(8, n8, 6.5, w.rest_s0);         // N-7..N -> N - 1/2
  set_grid_weights(w);
  cudaStreamSynchronize(e.stream);                 // tab lives on the host stack
}

// items of the level lists (build_lists): per star, at both register parities,
// ghost fill (2 per level and stage), the outer boundary after the last stage
// (1), restriction, child parity and parents' parity (1 each per level pair)
size_t litem_count(const std::vector<sacra_params> &ps) {
  const size_t S = ps.empty() ? 4 : (ps[0].rk == SACRA_RK4 ? 4 : 3);
  size_t n = 0;
  for (const sacra_params &p : ps) n += 2 * (2 * S * (size_t)p.n_levels + 1 + 3 * (size_t)(p.n_levels - 1));
  return n;
}

size_t engine_bytes(const std::vector<sacra_params> &ps) {
  size_t n = 0;
  int max_nx = 0;
  for (const sacra_params &p : ps) {
    n += star_bytes(&p);
    max_nx = std::max(max_nx, p.nx);
  }
  return n + round_up((size_t)(max_nx + 8) * (3 * kTabStride + kCartoonW) * 8, 256) + 256 /* dout */ + 256 /* nfb */ +
         256 /* tile counter */ +
         plan_bytes(ps) + round_up(litem_count(ps) * sizeof(LItem), 256);
}

sacra_status engine_init(Engine &e, const std::vector<sacra_params> &ps, void *stream, void *arena, size_t arena_bytes) {
  e.stream = (cudaStream_t)stream;
  if (cudaStreamCreateWithFlags(&e.up_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&e.up_start, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return SACRA_ERR_CUDA;
  }
  for (cudaEvent_t &ev : e.up_chunk)
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return SACRA_ERR_CUDA;
    }
  const size_t need = engine_bytes(ps);
  if (arena) {
    if (arena_bytes < need || ((uintptr_t)arena & 255)) return SACRA_ERR_OOM;
    e.arena = (char *)arena;
  } else {
    if (cudaMalloc(&e.arena, need) != cudaSuccess) {
      cudaGetLastError();
      return SACRA_ERR_OOM;
    }
    e.own_arena = true;
  }
  if (cudaMemsetAsync(e.arena, 0, need, e.stream) != cudaSuccess) {
    cudaGetLastError();
    return SACRA_ERR_CUDA;
  }
  fill_dev_params(&ps[0], &e.dp);
  e.S = ps[0].rk == SACRA_RK4 ? 4 : 3;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&e.sms, cudaDevAttrMultiProcessorCount, dev);
  if (e.sms < 1) e.sms = 1;
  char *p = e.arena;
  e.stars.resize(ps.size());
  int max_nx = 0;
  for (size_t i = 0; i < ps.size(); ++i) {
    Star &st = e.stars[i];
    st.prm = ps[i];
    fill_dev_params(&ps[i], &st.dp);
    st.lay = layout(&ps[i]);
    st.G = lockstep_levels(&ps[i]);
    init_star_levels(st, p);
    PwpTable tab;
    fill_pwp_table(&ps[i], &tab);
    cudaMemcpyAsync(st.pwp, &tab, sizeof(tab), cudaMemcpyHostToDevice, e.stream);
    if (cudaStreamSynchronize(e.stream) != cudaSuccess) return SACRA_ERR_CUDA;   // tab is on the stack
    if (st.dp.n_pieces > 1) st.dp.pwp = st.pwp;
    p += star_bytes(&ps[i]);
    max_nx = std::max(max_nx, ps[i].nx);
    for (int l = 0; l < ps[i].n_levels; ++l) {
      const int g = group_of(st, l);
      if (g >= (int)e.group_first.size()) e.group_first.push_back((int)e.slots.size());
      e.slots.push_back({(int)i, l});
      e.slot_group.push_back(g);
    }
  }
  e.ngroups = (int)e.group_first.size();
  e.dp.pwp = e.stars[0].dp.pwp;
  e.tab = (double *)p;
  e.tabw = e.tab + (size_t)(max_nx + 8) * 3 * kTabStride;
  p += round_up((size_t)(max_nx + 8) * (3 * kTabStride + kCartoonW) * 8, 256);
  e.dout = (double *)p;
  p += 256;
  e.nfb = (unsigned long long *)p;
  p += 256;
  e.tctr = (int *)p;
  p += 256;
  const size_t nl = e.slots.size();
  e.bl_dev = (BL *)p;
  p += round_up((2 * (size_t)e.S + 2) * nl * sizeof(BL), 256);
  e.tiles_dev = (Tile *)p;
  plan_caps(ps, &e.tiles_cap, &e.tune_cap);
  e.litems_dev = (LItem *)((char *)e.tiles_dev + round_up((e.tiles_cap + e.tune_cap) * sizeof(Tile), 256));
  e.litems_cap = litem_count(ps);
  for (Star &st : e.stars)
    for (int l = 0; l < st.prm.n_levels; ++l) st.lv[l].nfb = e.nfb;
  upload_tables(e, max_nx);
  const sacra_status s = upload_plan(e);
  if (s != SACRA_OK) return s;
  if (cudaStreamSynchronize(e.stream) != cudaSuccess || cudaGetLastError() != cudaSuccess) return SACRA_ERR_CUDA;
  return SACRA_OK;
}

void engine_free(Engine &e) {
  cudaStreamSynchronize(e.stream);
  if (e.up_stream) cudaStreamSynchronize(e.up_stream);
  drop_graphs(e);
  for (cudaEvent_t x : e.pool) cudaEventDestroy(x);
  if (e.up_start) cudaEventDestroy(e.up_start);
  for (cudaEvent_t x : e.up_chunk)
    if (x) cudaEventDestroy(x);
  if (e.up_stream) cudaStreamDestroy(e.up_stream);
  if (e.own_arena && e.arena) cudaFree(e.arena);
}

// ---------------------------------------------------------------- operations shared by both handles

sacra_status set_initial_data(Engine &e, int star, int level, int kind, const double *host, int n_fields) {
  if (star < 0 || star >= (int)e.stars.size()) return fail(e, SACRA_ERR_ARG, "bad star");
  Star &st = e.stars[star];
  if (level < 0 || level >= st.prm.n_levels || !host) return fail(e, SACRA_ERR_ARG, "bad level or buffer");
  if (n_fields != 30) return fail(e, SACRA_ERR_ARG, "n_fields must be 30");
  Lev &L = st.lv[level];
  const size_t np = (size_t)L.px * L.pz;
  // one pitched copy per group of planes (host planes are packed, device planes have stride P)
  if (kind == SACRA_PRIM_METRIC) {
    cudaMemcpy2DAsync(L.un, L.P * 8, host, np * 8, np * 8, NMET, cudaMemcpyHostToDevice, e.stream);
    cudaMemcpy2DAsync(L.prim, L.P * 8, host + (size_t)NMET * np, np * 8, np * 8, 5, cudaMemcpyHostToDevice, e.stream);
    run(e, K_PRIM2CONS, (long long)np, [&] { launch_prim2cons_all(L, st.dp, L.un, e.stream); });
  } else if (kind == SACRA_RAW) {
    // rows [1 - GH, nz + GH] in kUpChunks chunks: the copy of chunk c + 1 (upload
    // stream, after everything enqueued on the context's stream so far)
    // overlaps the recovery of chunk c (context stream, after chunk c arrived)
    cudaEventRecord(e.up_start, e.stream);
    cudaStreamWaitEvent(e.up_stream, e.up_start, 0);
    const int nrow = L.pz;
    for (int c = 0; c < Engine::kUpChunks; ++c) {
      const int r0 = nrow * c / Engine::kUpChunks, r1 = nrow * (c + 1) / Engine::kUpChunks;
      if (r1 <= r0) continue;
      const size_t off = (size_t)r0 * L.px;
      cudaMemcpy2DAsync(L.un + off, L.P * 8, host + off, np * 8, (size_t)(r1 - r0) * L.px * 8, NST,
                        cudaMemcpyHostToDevice, e.up_stream);
      cudaEventRecord(e.up_chunk[c], e.up_stream);
      cudaStreamWaitEvent(e.stream, e.up_chunk[c], 0);
      // padded row r is k = r - GH + 1
      run(e, K_C2P, (long long)(r1 - r0) * L.px, [&] {
        launch_c2p_region(L, st.dp, L.un, 1 - GH, L.nx + GH, r0 - GH + 1, r1 - GH, e.stream);
      });
    }
  } else {
    return fail(e, SACRA_ERR_ARG, "unknown kind");
  }
  cudaMemcpyAsync(L.us, L.un, (size_t)NST * L.P * 8, cudaMemcpyDeviceToDevice, e.stream);
  // the host buffer may be reused once it has been copied: wait for the copies
  // (RAW: the last chunk; the recovery goes on on the context's stream)
  const cudaError_t werr =
      kind == SACRA_RAW ? cudaStreamSynchronize(e.up_stream) : cudaStreamSynchronize(e.stream);
  if (werr != cudaSuccess) return cuda_check(e, "set_initial_data");
  st.have_data[level] = true;
  for (int l = 0; l < st.prm.n_levels; ++l) st.have_old[l] = false;   // no earlier time slice of the new data
  return cuda_check(e, "set_initial_data");
}

// all 30 padded state planes of one level to packed host planes (one pitched copy)
sacra_status read_level(Engine &e, int star, int level, int which, double *host, int n_fields) {
  if (star < 0 || star >= (int)e.stars.size()) return fail(e, SACRA_ERR_ARG, "bad star");
  Star &st = e.stars[star];
  if (level < 0 || level >= st.prm.n_levels || !host) return fail(e, SACRA_ERR_ARG, "bad level or buffer");
  if (n_fields != NST) return fail(e, SACRA_ERR_ARG, "n_fields must be 30");
  if (which != SACRA_STATE_STEP && which != SACRA_STATE_STAGE && which != SACRA_RHS)
    return fail(e, SACRA_ERR_ARG, "which must be a state or right-hand-side set");
  const Lev &L = st.lv[level];
  const size_t np = (size_t)L.px * L.pz;
  const double *src = which == SACRA_STATE_STEP ? L.un : (which == SACRA_STATE_STAGE ? L.us : L.rhs);
  cudaMemcpy2DAsync(host, np * 8, src, L.P * 8, np * 8, NST, cudaMemcpyDeviceToHost, e.stream);
  if (cudaStreamSynchronize(e.stream) != cudaSuccess) return cuda_check(e, "read_level");
  return cuda_check(e, "read_level");
}

sacra_status read_diag(Engine &e, sacra_diag *out);

// n_steps steps; with `diag` the first stage of each step also forms the
// diagnostics of the state at the start of the step, copied to diag[it]
sacra_status step(Engine &e, double dt, int n_steps, int use_graph, sacra_diag *diag = nullptr) {
  if (!ready(e)) return fail(e, SACRA_ERR_STATE, "initial data missing on some level");
  if (!(dt > 0) || n_steps < 0) return fail(e, SACRA_ERR_ARG, "bad dt or n_steps");
  if (diag && e.ngroups > 1) return fail(e, SACRA_ERR_STATE, "diagnostics inside the step need a lockstep context");
  for (int it = 0; it < n_steps; ++it) {
    e.stage0_diag = diag != nullptr;
    if (!use_graph || !steady(e)) {
      enqueue_step(e, dt);
    } else {
      const int gi = 2 * e.parity + (diag ? 1 : 0);
      if (!e.gexec[gi] || e.gdt[gi] != dt) {
        if (e.gexec[gi]) { cudaGraphExecDestroy(e.gexec[gi]); e.gexec[gi] = nullptr; }
        cudaGraph_t g;
        const long long before = e.launches;
        if (cudaStreamBeginCapture(e.stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
          e.stage0_diag = false;
          return cuda_check(e, "graph capture (the stream must be a non-default stream)");
        }
        e.capturing = true;
        enqueue_step(e, dt);       // swaps the registers on the host side (a sub-cycled
        e.capturing = false;       // level swaps an even number of times per step)
        e.stage0_diag = false;
        if (cudaStreamEndCapture(e.stream, &g) != cudaSuccess) return cuda_check(e, "graph capture");
        e.glaunch[gi] = e.launches - before;
        e.launches = before;
        swap_group(e, 0);          // undo: the graph has not run yet
        if (cudaGraphInstantiate(&e.gexec[gi], g, 0) != cudaSuccess) {
          cudaGraphDestroy(g);
          return cuda_check(e, "graph instantiate");
        }
        cudaGraphDestroy(g);
        e.gdt[gi] = dt;
      }
      if (cudaGraphLaunch(e.gexec[gi], e.stream) != cudaSuccess) {
        e.stage0_diag = false;
        return cuda_check(e, "graph launch");
      }
      e.launches += e.glaunch[gi];
      for (Star &st : e.stars) st.dt_step = dt;
      swap_group(e, 0);
    }
    e.stage0_diag = false;
    if (diag) {
      const sacra_status r = read_diag(e, &diag[it]);
      if (r != SACRA_OK) return r;
    }
  }
  return cuda_check(e, "step");
}

sacra_status read_state(Engine &e, int star, int level, int which, int field, double *host, size_t n) {
  if (star < 0 || star >= (int)e.stars.size()) return fail(e, SACRA_ERR_ARG, "bad star");
  Star &st = e.stars[star];
  if (level < 0 || level >= st.prm.n_levels || !host) return fail(e, SACRA_ERR_ARG, "bad level or buffer");
  Lev &L = st.lv[level];
  const size_t np = (size_t)L.px * L.pz;
  const double *src = nullptr;
  std::vector<double> tmp;
  if (which == SACRA_STATE_STEP || which == SACRA_STATE_STAGE || which == SACRA_RHS) {
    if (field < 0 || field >= NST) return fail(e, SACRA_ERR_ARG, "bad field");
    const double *base = which == SACRA_STATE_STEP ? L.un : (which == SACRA_STATE_STAGE ? L.us : L.rhs);
    src = base + (size_t)field * L.P;
  } else if (which == SACRA_PRIMS) {
    if (field < 0 || field >= NPRIM) return fail(e, SACRA_ERR_ARG, "bad field");
    src = L.prim + (size_t)field * L.P;
  } else if (which != SACRA_STATUS) {
    return fail(e, SACRA_ERR_ARG, "unknown plane");
  }
  tmp.resize(np);
  if (which == SACRA_STATUS) {
    std::vector<int> sv(np);
    cudaMemcpyAsync(sv.data(), L.status, np * 4, cudaMemcpyDeviceToHost, e.stream);
    if (cudaStreamSynchronize(e.stream) != cudaSuccess) return cuda_check(e, "read_state");
    for (size_t i = 0; i < np; ++i) tmp[i] = sv[i];
  } else {
    cudaMemcpyAsync(tmp.data(), src, np * 8, cudaMemcpyDeviceToHost, e.stream);
    if (cudaStreamSynchronize(e.stream) != cudaSuccess) return cuda_check(e, "read_state");
  }
  if (n == np) {
    memcpy(host, tmp.data(), np * 8);
  } else if (n == (size_t)L.nx * L.nz) {
    for (int k = 1; k <= L.nz; ++k) memcpy(host + (size_t)(k - 1) * L.nx, tmp.data() + cid(L, 1, k), (size_t)L.nx * 8);
  } else {
    return fail(e, SACRA_ERR_ARG, "n must be nx*nz or px*pz");
  }
  return cuda_check(e, "read_state");
}

// the constraint and conservation diagnostics of the star's current state
// (Sec. II.F.1): per-level partial sums, then one fixed-order final sum into
// e.dout.  own_derivs: run the cartoon and derivative passes first; without
// it the level scratch must already hold the derivatives of this state (the
// first stage of a step has just formed them).
void enqueue_diag(Engine &e, Star &st, bool own_derivs) {
  const int L = st.prm.n_levels;
  int slot = 0;
  for (int l = 0; l < L; ++l) {
    Lev &lv = st.lv[l];
    const long long cells = (long long)lv.nx * lv.nz;
    double *ds = reinterpret_cast<double *>(st.ds[l]);
    if (own_derivs && st.prm.evolve_spacetime) {
      run(e, K_CARTOON, (long long)(lv.nx + 7) * (lv.nz + 10), [&] { launch_cartoon(lv, st.dp, lv.un, e.tab, kTabStride, e.tabw, e.stream); });
      run(e, K_Z4C_DERIVS, cells, [&] { launch_z4c_derivs(lv, st.dp, lv.un, ds, lv.nx, lv.nz, e.stream); });
    }
    const int sl = slot;
    // in a step, the pointwise pass has also stored the Ricci scalar (in the
    // mixed form the FP32 value its own algebra used)
    const double *rs = (!own_derivs && st.prm.evolve_spacetime) ? ds + (size_t)z4c_ricci_plane() * lv.P : nullptr;
    run(e, K_DIAG, cells, [&] { launch_diag(lv, st.dp, ds, l < L - 1, st.prm.evolve_spacetime, st.part, sl, e.stream, rs); });
    slot += diag_blocks(lv);
  }
  run(e, K_DIAG_FINAL, slot, [&] { launch_diag_final(st.part, slot, e.dout, e.stream); });
}

// copy the final sums and the fallback counter to the host (waits for the stream)
sacra_status read_diag(Engine &e, sacra_diag *out) {
  double h[9];
  unsigned long long nfb = 0;
  cudaMemcpyAsync(h, e.dout, sizeof(h), cudaMemcpyDeviceToHost, e.stream);
  cudaMemcpyAsync(&nfb, e.nfb, sizeof(nfb), cudaMemcpyDeviceToHost, e.stream);
  if (cudaStreamSynchronize(e.stream) != cudaSuccess) return cuda_check(e, "constraints");
  out->H_L2 = sqrt(h[0] / h[4]);
  for (int a = 0; a < 3; ++a) out->M_L2[a] = sqrt(h[1 + a] / h[4]);
  out->Mb = h[5];
  out->J = h[6];
  out->rho_max = h[7];
  out->n_c2p_fail = h[8];
  out->n_fallback = (double)nfb;
  return cuda_check(e, "constraints");
}

sacra_status constraints(Engine &e, int star, sacra_diag *out) {
  if (star < 0 || star >= (int)e.stars.size() || !out) return fail(e, SACRA_ERR_ARG, "bad star or output");
  if (!ready(e)) return fail(e, SACRA_ERR_STATE, "initial data missing on some level");
  Star &st = e.stars[star];
  enqueue_fill(e, st, 0, 0.0);
  enqueue_diag(e, st, true);
  return read_diag(e, out);
}

sacra_status profile_get(Engine &e, int idx, char *name, size_t name_len, double *total_ms, long long *launches,
                         long long *cells) {
  if (idx < 0 || idx >= K_COUNT || !name || name_len == 0) return SACRA_ERR_ARG;
  if (cudaStreamSynchronize(e.stream) != cudaSuccess) return cuda_check(e, "profile_get");
  double ms = 0.0;
  long long n = 0, cl = 0;
  for (const ProfRec &r : e.recs) {
    if (r.kid != idx) continue;
    float t = 0.f;
    cudaEventElapsedTime(&t, r.a, r.b);
    ms += t;
    ++n;
    cl += r.cells;
  }
  snprintf(name, name_len, "%s", kKidName[idx]);
  if (total_ms) *total_ms = ms;
  if (launches) *launches = n;
  if (cells) *cells = cl;
  return cuda_check(e, "profile_get");
}

sacra_status get_tuning(const Engine &e, int kind, int *tile_x, int *tile_y, int *blocks_per_sm) {
  if (kind < 0 || kind >= B_NKIND) return SACRA_ERR_ARG;
  const Shape sh = kind_shape(e, kind);
  if (tile_x) *tile_x = sh.x;
  if (tile_y) *tile_y = sh.y;
  if (blocks_per_sm) *blocks_per_sm = e.cfg[kind].blocks_per_sm;
  return SACRA_OK;
}

// pins one kind's launch configuration to a candidate of the autotuner
sacra_status set_tuning(Engine &e, int kind, int tile_x, int tile_y, int blocks_per_sm) {
  if (kind < 0 || kind >= B_NKIND) return SACRA_ERR_ARG;
  bool shape_ok = false, m_ok = false;
  if (fixed_shape(e, kind)) {
    const Shape f = kind_shape(e, kind);
    shape_ok = f.x == tile_x && f.y == tile_y;
  } else if (max_threads(kind) >= 256) {
    for (const Shape &sh : kShapes256) shape_ok = shape_ok || (sh.x == tile_x && sh.y == tile_y);
  } else {
    for (const Shape &sh : kShapes128) shape_ok = shape_ok || (sh.x == tile_x && sh.y == tile_y);
  }
  for (int m : kBlocksPerSm) m_ok = m_ok || m == blocks_per_sm;
  if (!shape_ok || !m_ok) return SACRA_ERR_ARG;
  drop_graphs(e);
  if (!fixed_shape(e, kind)) e.cfg[kind].shape = Shape{tile_x, tile_y};
  e.cfg[kind].blocks_per_sm = blocks_per_sm;
  const sacra_status st = upload_plan(e);
  if (st != SACRA_OK) return st;
  return cuda_check(e, "set_tuning");
}

sacra_status set_profile(Engine &e, int enable) {
  e.prof = enable != 0;
  e.recs.clear();
  e.pool_used = 0;
  return SACRA_OK;
}

sacra_status sync(Engine &e) {
  if (cudaStreamSynchronize(e.stream) != cudaSuccess) return cuda_check(e, "sync");
  return cuda_check(e, "sync");
}

// ---- learned seed of the primitive recovery

unsigned long long *c2p_counters(Engine &e) { return e.nfb + 1; }   // 4 counters next to the fallback count
unsigned long long *collect_counter(Engine &e) { return e.nfb + 8; }

sacra_status set_mlp(Engine &e, const void *dev_net) {
  const MlpNet *net = reinterpret_cast<const MlpNet *>(dev_net);
  e.dp.mlp = net;
  for (Star &st : e.stars) st.dp.mlp = net;
  drop_graphs(e);
  return upload_plan(e);
}

sacra_status set_counting(Engine &e, int on) {
  unsigned long long *c = on ? c2p_counters(e) : nullptr;
  e.dp.c2p_stats = c;
  for (Star &st : e.stars) st.dp.c2p_stats = c;
  if (on) cudaMemsetAsync(c2p_counters(e), 0, 4 * sizeof(unsigned long long), e.stream);
  drop_graphs(e);
  return upload_plan(e);
}

sacra_status get_counts(Engine &e, long long out[4], int reset) {
  unsigned long long h[4];
  cudaMemcpyAsync(h, c2p_counters(e), sizeof(h), cudaMemcpyDeviceToHost, e.stream);
  if (reset) cudaMemsetAsync(c2p_counters(e), 0, sizeof(h), e.stream);
  if (cudaStreamSynchronize(e.stream) != cudaSuccess) return cuda_check(e, "c2p counts");
  for (int a = 0; a < 4; ++a) out[a] = (long long)h[a];
  return cuda_check(e, "c2p counts");
}

sacra_status mlp_collect(Engine &e, float *dev_out, long long cap, long long *n) {
  if (!dev_out || cap < 0 || !n) return fail(e, SACRA_ERR_ARG, "bad buffer");
  if (!ready(e)) return fail(e, SACRA_ERR_STATE, "initial data missing on some level");
  cudaMemsetAsync(collect_counter(e), 0, sizeof(unsigned long long), e.stream);
  for (Star &st : e.stars)
    for (int l = 0; l < st.prm.n_levels; ++l)   // the level's derivative scratch holds the block counts
      launch_mlp_collect(st.lv[l], st.dp, dev_out, cap, collect_counter(e), st.ds[l], e.stream);
  unsigned long long h = 0;
  cudaMemcpyAsync(&h, collect_counter(e), sizeof(h), cudaMemcpyDeviceToHost, e.stream);
  if (cudaStreamSynchronize(e.stream) != cudaSuccess) return cuda_check(e, "mlp_collect");
  *n = std::min<long long>((long long)h, cap);
  return cuda_check(e, "mlp_collect");
}

// a batch's stars share one launch group per stage, so none of them sub-cycles
bool params_ok(const sacra_params *per_star, int n) {
  if (!per_star || n < 1) return false;
  std::string why;
  for (int i = 0; i < n; ++i) {
    if (!valid(&per_star[i], &why) || !compatible(&per_star[i], &per_star[0])) return false;
    if (n > 1 && lockstep_levels(&per_star[i]) < per_star[i].n_levels) return false;
  }
  return true;
}

}  // namespace

extern "C" {

// ---------------------------------------------------------------- one star

sacra_status sacra_arena_bytes(const sacra_params *p, size_t *bytes) {
  if (!bytes || !params_ok(p, 1)) return SACRA_ERR_ARG;
  *bytes = engine_bytes({*p});
  return SACRA_OK;
}

sacra_status sacra_init_grid(const sacra_params *p, void *cuda_stream, void *arena, size_t arena_bytes,
                             sacra_ctx **out) {
  if (!out) return SACRA_ERR_ARG;
  *out = nullptr;
  if (!params_ok(p, 1)) return SACRA_ERR_ARG;
  sacra_ctx *c = new sacra_ctx();
  const sacra_status s = engine_init(c->e, {*p}, cuda_stream, arena, arena_bytes);
  if (s != SACRA_OK) {
    engine_free(c->e);
    delete c;
    return s;
  }
  *out = c;
  return SACRA_OK;
}

sacra_status sacra_set_initial_data(sacra_ctx *c, int level, int kind, const double *host, int n_fields) {
  if (!c) return SACRA_ERR_ARG;
  return set_initial_data(c->e, 0, level, kind, host, n_fields);
}

sacra_status sacra_regrid_ghosts(sacra_ctx *c, int what, int stage, double dt) {
  if (!c) return SACRA_ERR_ARG;
  Engine &e = c->e;
  if (!ready(e)) return fail(e, SACRA_ERR_STATE, "initial data missing on some level");
  if (e.ngroups > 1) return fail(e, SACRA_ERR_STATE, "stage-wise calls need a lockstep context");
  if (what == SACRA_FILL) {
    if (stage < 0 || stage >= e.S) return fail(e, SACRA_ERR_ARG, "bad stage");
    enqueue_fill(e, e.stars[0], stage, dt);
  } else if (what == SACRA_RESTRICT_REFLUX) {
    enqueue_restrict(e, e.stars[0]);
  } else {
    return fail(e, SACRA_ERR_ARG, "unknown regrid request");
  }
  return cuda_check(e, "regrid_ghosts");
}

sacra_status sacra_rk_stage(sacra_ctx *c, int stage, double dt) {
  if (!c) return SACRA_ERR_ARG;
  Engine &e = c->e;
  if (!ready(e)) return fail(e, SACRA_ERR_STATE, "initial data missing on some level");
  if (e.ngroups > 1) return fail(e, SACRA_ERR_STATE, "stage-wise calls need a lockstep context");
  if (stage < 0 || stage >= e.S || !(dt > 0)) return fail(e, SACRA_ERR_ARG, "bad stage or dt");
  enqueue_stage(e, stage, dt);
  return cuda_check(e, "rk_stage");
}

sacra_status sacra_step(sacra_ctx *c, double dt, int n_steps, int use_graph) {
  if (!c) return SACRA_ERR_ARG;
  return step(c->e, dt, n_steps, use_graph);
}

sacra_status sacra_step_constraints(sacra_ctx *c, double dt, int n_steps, int use_graph, sacra_diag *out) {
  if (!c) return SACRA_ERR_ARG;
  if (!out && n_steps > 0) return fail(c->e, SACRA_ERR_ARG, "out must hold n_steps diagnostics");
  return step(c->e, dt, n_steps, use_graph, out);
}

sacra_status sacra_read_state(sacra_ctx *c, int level, int which, int field, double *host, size_t n) {
  if (!c) return SACRA_ERR_ARG;
  return read_state(c->e, 0, level, which, field, host, n);
}

sacra_status sacra_read_level(sacra_ctx *c, int level, int which, double *host_planes, int n_fields) {
  if (!c) return SACRA_ERR_ARG;
  return read_level(c->e, 0, level, which, host_planes, n_fields);
}

sacra_status sacra_constraints(sacra_ctx *c, sacra_diag *out) {
  if (!c || !out) return SACRA_ERR_ARG;
  return constraints(c->e, 0, out);
}

sacra_status sacra_sync(sacra_ctx *c) { return c ? sync(c->e) : SACRA_ERR_ARG; }

long long sacra_launch_count(const sacra_ctx *c) { return c ? c->e.launches : -1; }

sacra_status sacra_profile(sacra_ctx *c, int enable) { return c ? set_profile(c->e, enable) : SACRA_ERR_ARG; }

sacra_status sacra_profile_get(sacra_ctx *c, int idx, char *name, size_t name_len, double *total_ms,
                               long long *launches, long long *cells) {
  if (!c) return SACRA_ERR_ARG;
  return profile_get(c->e, idx, name, name_len, total_ms, launches, cells);
}

sacra_status sacra_tune(sacra_ctx *c, int reps) { return c ? tune(c->e, reps) : SACRA_ERR_ARG; }

sacra_status sacra_get_tuning(const sacra_ctx *c, int kind, int *tile_x, int *tile_y, int *blocks_per_sm) {
  return c ? get_tuning(c->e, kind, tile_x, tile_y, blocks_per_sm) : SACRA_ERR_ARG;
}

sacra_status sacra_set_tuning(sacra_ctx *c, int kind, int tile_x, int tile_y, int blocks_per_sm) {
  return c ? set_tuning(c->e, kind, tile_x, tile_y, blocks_per_sm) : SACRA_ERR_ARG;
}

size_t sacra_mlp_bytes(void) { return sizeof(MlpNet); }

sacra_status sacra_mlp_collect(sacra_ctx *c, float *dev_tuples, long long capacity, long long *n) {
  return c ? mlp_collect(c->e, dev_tuples, capacity, n) : SACRA_ERR_ARG;
}

sacra_status sacra_mlp_train(const float *dev_tuples, long long n, int steps, int batch_blocks, float lr,
                             unsigned long long seed, float kmin, void *dev_net, float *host_loss, float *host_report,
                             void *cuda_stream) {
  const int rc = mlp_train(dev_tuples, n, steps, batch_blocks, lr, seed, kmin, reinterpret_cast<MlpNet *>(dev_net),
                           host_loss, host_report, (cudaStream_t)cuda_stream);
  if (rc == -1) return SACRA_ERR_ARG;
  if (rc == -3) return SACRA_ERR_OOM;
  return rc == 0 && cudaGetLastError() == cudaSuccess ? SACRA_OK : SACRA_ERR_CUDA;
}

sacra_status sacra_mlp_grad(const float *dev_tuples, long long n, const void *dev_net, float *host_grad,
                            float *host_loss, void *cuda_stream) {
  const int rc = mlp_grad(dev_tuples, n, reinterpret_cast<const MlpNet *>(dev_net), host_grad, host_loss,
                          (cudaStream_t)cuda_stream);
  if (rc == -1) return SACRA_ERR_ARG;
  if (rc == -3) return SACRA_ERR_OOM;
  return rc == 0 && cudaGetLastError() == cudaSuccess ? SACRA_OK : SACRA_ERR_CUDA;
}

sacra_status sacra_set_mlp(sacra_ctx *c, const void *dev_net) { return c ? set_mlp(c->e, dev_net) : SACRA_ERR_ARG; }

sacra_status sacra_c2p_counting(sacra_ctx *c, int enable) { return c ? set_counting(c->e, enable) : SACRA_ERR_ARG; }

sacra_status sacra_c2p_counts(sacra_ctx *c, long long *out4, int reset) {
  return c && out4 ? get_counts(c->e, out4, reset) : SACRA_ERR_ARG;
}

void sacra_destroy(sacra_ctx *c) {
  if (!c) return;
  engine_free(c->e);
  delete c;
}

const char *sacra_last_error(const sacra_ctx *c) { return c ? c->e.err.c_str() : "null context"; }

// ---------------------------------------------------------------- a batch of stars

sacra_status sacra_batch_arena_bytes(const sacra_params *per_star, int n_stars, size_t *bytes) {
  if (!bytes || !params_ok(per_star, n_stars)) return SACRA_ERR_ARG;
  *bytes = engine_bytes(std::vector<sacra_params>(per_star, per_star + n_stars));
  return SACRA_OK;
}

sacra_status sacra_init_batch(const sacra_params *per_star, int n_stars, void *cuda_stream, void *arena,
                              size_t arena_bytes, sacra_batch **out) {
  if (!out) return SACRA_ERR_ARG;
  *out = nullptr;
  if (!params_ok(per_star, n_stars)) return SACRA_ERR_ARG;
  sacra_batch *b = new sacra_batch();
  const sacra_status s =
      engine_init(b->e, std::vector<sacra_params>(per_star, per_star + n_stars), cuda_stream, arena, arena_bytes);
  if (s != SACRA_OK) {
    engine_free(b->e);
    delete b;
    return s;
  }
  *out = b;
  return SACRA_OK;
}

sacra_status sacra_batch_set_initial_data(sacra_batch *b, int star, int level, int kind, const double *host,
                                          int n_fields) {
  return b ? set_initial_data(b->e, star, level, kind, host, n_fields) : SACRA_ERR_ARG;
}

sacra_status sacra_batch_step(sacra_batch *b, double dt, int n_steps, int use_graph) {
  return b ? step(b->e, dt, n_steps, use_graph) : SACRA_ERR_ARG;
}

sacra_status sacra_batch_read_state(sacra_batch *b, int star, int level, int which, int field, double *host,
                                    size_t n) {
  return b ? read_state(b->e, star, level, which, field, host, n) : SACRA_ERR_ARG;
}

sacra_status sacra_batch_constraints(sacra_batch *b, int star, sacra_diag *out) {
  return b ? constraints(b->e, star, out) : SACRA_ERR_ARG;
}

sacra_status sacra_batch_tune(sacra_batch *b, int reps) { return b ? tune(b->e, reps) : SACRA_ERR_ARG; }

sacra_status sacra_batch_get_tuning(const sacra_batch *b, int kind, int *tile_x, int *tile_y, int *blocks_per_sm) {
  return b ? get_tuning(b->e, kind, tile_x, tile_y, blocks_per_sm) : SACRA_ERR_ARG;
}

sacra_status sacra_batch_set_tuning(sacra_batch *b, int kind, int tile_x, int tile_y, int blocks_per_sm) {
  return b ? set_tuning(b->e, kind, tile_x, tile_y, blocks_per_sm) : SACRA_ERR_ARG;
}

sacra_status sacra_batch_sync(sacra_batch *b) { return b ? sync(b->e) : SACRA_ERR_ARG; }

long long sacra_batch_launch_count(const sacra_batch *b) { return b ? b->e.launches : -1; }

sacra_status sacra_batch_profile(sacra_batch *b, int enable) { return b ? set_profile(b->e, enable) : SACRA_ERR_ARG; }

sacra_status sacra_batch_profile_get(sacra_batch *b, int idx, char *name, size_t name_len, double *total_ms,
                                     long long *launches, long long *cells) {
  return b ? profile_get(b->e, idx, name, name_len, total_ms, launches, cells) : SACRA_ERR_ARG;
}

sacra_status sacra_batch_set_mlp(sacra_batch *b, const void *dev_net) {
  return b ? set_mlp(b->e, dev_net) : SACRA_ERR_ARG;
}

sacra_status sacra_batch_mlp_collect(sacra_batch *b, float *dev_tuples, long long capacity, long long *n) {
  return b ? mlp_collect(b->e, dev_tuples, capacity, n) : SACRA_ERR_ARG;
}

void sacra_batch_destroy(sacra_batch *b) {
  if (!b) return;
  engine_free(b->e);
  delete b;
}

const char *sacra_batch_last_error(const sacra_batch *b) { return b ? b->e.err.c_str() : "null batch"; }

}  // extern "C"
