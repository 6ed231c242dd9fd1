// C ABI of the SACRA-2D hot path (include/sacra2d.h): context, device arena,
// the stage sequence of Sec. II.D (lockstep levels), CUDA-graph replay of
// whole steps.  All arithmetic runs in the kernels of hydro.cu, z4c.cu and
// grid.cu; the host only orders launches and computes interpolation weights.
#include <math.h>
#include <stdio.h>
#include <string.h>

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

struct Layout {
  size_t P;          // plane stride (doubles), multiple of 32
  int rw;            // flux register row width
  size_t per_level;  // bytes
  size_t shared;     // bytes after the levels
  size_t ds_off, dy_off, dyy_off, tab_off, part_off, dout_off, nfb_off;
  int n_part;        // diag partial blocks (all levels)
};

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
  return true;
}

Layout layout(const sacra_params *p) {
  Layout o;
  const size_t px = p->nx + 2 * GH, pz = p->nz + 2 * GH;
  o.P = round_up(px * pz, 32);
  o.rw = (p->nx > p->nz ? p->nx : p->nz) + 2;
  const size_t rwp = round_up((size_t)o.rw, 32);
  const size_t planes = 4 * NST + NPRIM + 2 * NCONS;
  o.per_level = planes * o.P * 8 + o.P * 4 /* status */ + 4 * NCONS * rwp * 8;
  o.per_level = round_up(o.per_level, 256);
  size_t off = 0;
  o.ds_off = off; off += round_up((size_t)z4c_scratch_planes() * o.P * 8, 256);
  o.dy_off = off; off += round_up((size_t)NMET * o.P * 8, 256);
  o.dyy_off = off; off += round_up((size_t)NMET * o.P * 8, 256);
  o.tab_off = off; off += round_up((size_t)(p->nx + 8) * 3 * kTabStride * 8, 256);
  o.n_part = p->n_levels * ((p->nx * p->nz + 127) / 128);
  o.part_off = off; off += round_up((size_t)o.n_part * 9 * 8, 256);
  o.dout_off = off; off += 256;
  o.nfb_off = off; off += 256;
  o.shared = off;
  return o;
}

}  // namespace

// kernel kinds for launch counting and the optional per-kernel profile
enum Kid {
  K_OUTFLOW, K_OUTER, K_PROLONG, K_PARITY_X, K_PARITY_Z, K_FLUX_X, K_FLUX_Z, K_HYDRO_DIV, K_CARTOON, K_Z4C_DERIVS,
  K_Z4C_POINT, K_RK_UPDATE, K_RESTRICT, K_REFLUX, K_C2P, K_PRIM2CONS, K_DIAG, K_DIAG_FINAL, K_COUNT
};
static const char *kKidName[K_COUNT] = {"k_outflow", "k_outer", "k_prolong", "k_parity_x", "k_parity_z", "k_flux_x",
                                        "k_flux_z", "k_hydro_rhs", "k_cartoon", "k_z4c_derivs", "k_z4c_point",
                                        "k_rk_update", "k_restrict", "k_reflux", "k_c2p_region", "k_prim2cons_all",
                                        "k_diag", "k_diag_final"};

struct ProfRec {
  int kid;
  cudaEvent_t a, b;
  long long cells;
};

struct sacra_ctx {
  sacra_params prm;
  DevParams dp;
  Layout lay;
  cudaStream_t stream = nullptr;
  char *arena = nullptr;
  bool own_arena = false;
  Lev lv[kMaxLevels];
  double *ds = nullptr, *tab = nullptr, *part = nullptr, *dout = nullptr;
  unsigned long long *nfb = nullptr;
  double dt_step = 0.0;
  bool have_data[kMaxLevels] = {};
  long long launches = 0;
  std::string err;
  // graph replay: one graph per parity of the register swap
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  double gdt[2] = {0.0, 0.0};
  long long glaunch[2] = {0, 0};
  int parity = 0;    // number of register swaps mod 2
  bool capturing = false;
  // per-kernel profile (eager launches only)
  bool prof = false;
  std::vector<ProfRec> recs;
  std::vector<cudaEvent_t> pool;
  size_t pool_used = 0;
};

namespace {

sacra_status fail(sacra_ctx *c, sacra_status s, const std::string &m) {
  if (c) c->err = m;
  return s;
}

sacra_status cuda_check(sacra_ctx *c, const char *where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(c, SACRA_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
  return SACRA_OK;
}

cudaEvent_t pool_event(sacra_ctx *c) {
  if (c->pool_used == c->pool.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    c->pool.push_back(e);
  }
  return c->pool[c->pool_used++];
}

// every kernel launch goes through here: count it, and bracket it with
// events when profiling (not while a graph is being captured)
template <class F>
void run(sacra_ctx *c, Kid k, long long cells, F &&launch) {
  if (c->prof && !c->capturing) {
    ProfRec r{(int)k, pool_event(c), pool_event(c), cells};
    cudaEventRecord(r.a, c->stream);
    launch();
    cudaEventRecord(r.b, c->stream);
    c->recs.push_back(r);
  } else {
    launch();
  }
  ++c->launches;
}

int n_stages(const sacra_ctx *c) { return c->prm.rk == SACRA_RK4 ? 4 : 3; }
double stage_c(const sacra_ctx *c, int s) {
  static const double c4[4] = {0.0, 0.5, 0.5, 1.0}, c3[3] = {0.0, 1.0, 0.5};
  return c->prm.rk == SACRA_RK4 ? c4[s] : c3[s];
}
double stage_b(const sacra_ctx *c, int s) {
  static const double b4[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0}, b3[3] = {1.0 / 6.0, 1.0 / 6.0, 2.0 / 3.0};
  return c->prm.rk == SACRA_RK4 ? b4[s] : b3[s];
}
double *stage_state(sacra_ctx *c, int l, int s) { return s == 0 ? c->lv[l].un : c->lv[l].us; }

void region(const sacra_ctx *c, int l, int s, int *jmax, int *kmax) {
  const int ext = (l > 0 && s < n_stages(c) - 1) ? 4 : 0;
  *jmax = c->prm.nx + ext;
  *kmax = c->prm.nz + ext;
}

void enqueue_parity(sacra_ctx *c, int l, double *U) {
  const Lev &L = c->lv[l];
  run(c, K_PARITY_X, 8LL * (L.nz + GH), [&] { launch_parity_x(L, U, c->stream); });
  run(c, K_PARITY_Z, 8LL * (L.nx + 2 * GH), [&] { launch_parity_z(L, U, c->stream); });
}

void enqueue_fill(sacra_ctx *c, int s, double dt) {
  for (int l = 0; l < c->prm.n_levels; ++l) {
    double *U = stage_state(c, l, s);
    const Lev &L = c->lv[l];
    if (c->prm.geometry == SACRA_PLANAR) {
      run(c, K_OUTFLOW, (long long)L.px * L.pz, [&] { launch_outflow(L, U, c->stream); });
      continue;
    }
    if (l == 0) {
      run(c, K_OUTER, (long long)(L.nx + GH) * (L.nz + GH) - (long long)L.nx * L.nz,
          [&] { launch_outer(L, L.un, U, stage_c(c, s) * dt, c->stream); });
    } else {
      double *Up = stage_state(c, l - 1, s);
      run(c, K_PROLONG, prolong_cells(L, s == 0), [&] { launch_prolong(L, c->lv[l - 1], c->dp, U, Up, s == 0, c->stream); });
      ++c->launches;   // the prolongation is two kernels
    }
    enqueue_parity(c, l, U);
  }
}

void swap_registers(sacra_ctx *c) {
  for (int l = 0; l < c->prm.n_levels; ++l) {
    double *t = c->lv[l].un;
    c->lv[l].un = c->lv[l].us;
    c->lv[l].us = t;
  }
  c->parity ^= 1;
}

void enqueue_stage(sacra_ctx *c, int s, double dt) {
  const int S = n_stages(c);
  const int L = c->prm.n_levels;
  if (s == 0) {
    c->dt_step = dt;
    for (int l = 0; l < L; ++l)
      cudaMemsetAsync(c->lv[l].freg, 0, (size_t)4 * NCONS * c->lv[l].rw * sizeof(double), c->stream);
  }
  for (int l = 0; l < L; ++l) {
    Lev &lv = c->lv[l];
    double *U = stage_state(c, l, s);
    int jmax, kmax;
    region(c, l, s, &jmax, &kmax);
    const long long cells = (long long)jmax * kmax;
    const double wb = stage_b(c, s);
    const int hc = l < L - 1, hp = l > 0;
    run(c, K_FLUX_X, cells, [&] { launch_flux_x(lv, c->dp, U, jmax, kmax, wb, hc, hp, c->stream); });
    run(c, K_FLUX_Z, cells, [&] { launch_flux_z(lv, c->dp, U, jmax, kmax, wb, hc, hp, c->stream); });
    run(c, K_HYDRO_DIV, cells, [&] { launch_hydro_div(lv, c->dp, U, jmax, kmax, c->stream); });
    if (c->prm.evolve_spacetime) {
      if (c->prm.geometry == SACRA_CYLINDRICAL)
        run(c, K_CARTOON, (long long)(lv.nx + 7) * (lv.nz + 10), [&] { launch_cartoon(lv, c->dp, U, c->tab, kTabStride, c->stream); });
      run(c, K_Z4C_DERIVS, cells, [&] { launch_z4c_derivs(lv, c->dp, U, c->ds, jmax, kmax, c->stream); });
      run(c, K_Z4C_POINT, cells, [&] { launch_z4c_point(lv, c->dp, U, c->ds, jmax, kmax, c->stream); });
    }
    run(c, K_RK_UPDATE, cells, [&] { launch_rk_update(lv, c->dp, U, s, dt, jmax, kmax, c->stream); });
  }
  if (s == S - 1) {
    if (c->prm.geometry == SACRA_CYLINDRICAL) {
      const Lev &L0 = c->lv[0];
      run(c, K_OUTER, (long long)(L0.nx + GH) * (L0.nz + GH) - (long long)L0.nx * L0.nz,
          [&] { launch_outer(L0, L0.un, L0.us, dt, c->stream); });
    }
    swap_registers(c);
  }
}

void enqueue_restrict(sacra_ctx *c) {
  const int L = c->prm.n_levels;
  if (L < 2) return;
  for (int l = L - 1; l >= 1; --l) {
    Lev &C = c->lv[l], &Pa = c->lv[l - 1];
    enqueue_parity(c, l, C.un);
    const int nh = Pa.nx / 2;
    run(c, K_RESTRICT, (long long)nh * nh, [&] { launch_restrict(C, Pa, c->stream); });
    run(c, K_REFLUX, 2LL * nh, [&] { launch_reflux(C, Pa, c->dt_step, c->stream); });
    // the restricted cells [1, N/2]^2 and the refluxed strips next to them (not the corner)
    run(c, K_C2P, (long long)(nh + 1) * (nh + 1) - 1,
        [&] { launch_c2p_region(Pa, c->dp, Pa.un, 1, nh + 1, 1, nh + 1, c->stream, 1); });
  }
  // the parents' axis/equator ghosts mirror their restricted interiors
  for (int l = 0; l < L - 1; ++l) enqueue_parity(c, l, c->lv[l].un);
}

void enqueue_step(sacra_ctx *c, double dt) {
  const int S = n_stages(c);
  for (int s = 0; s < S; ++s) {
    enqueue_fill(c, s, dt);
    enqueue_stage(c, s, dt);
  }
  enqueue_restrict(c);
}

}  // namespace

extern "C" {

sacra_status sacra_arena_bytes(const sacra_params *p, size_t *bytes) {
  std::string why;
  if (!bytes || !valid(p, &why)) return SACRA_ERR_ARG;
  const Layout o = layout(p);
  *bytes = o.per_level * p->n_levels + o.shared;
  return SACRA_OK;
}

sacra_status sacra_init_grid(const sacra_params *p, void *cuda_stream, void *arena, size_t arena_bytes,
                             sacra_ctx **out) {
  if (!out) return SACRA_ERR_ARG;
  *out = nullptr;
  std::string why;
  if (!valid(p, &why)) return SACRA_ERR_ARG;
  sacra_ctx *c = new sacra_ctx();
  c->prm = *p;
  c->lay = layout(p);
  c->stream = (cudaStream_t)cuda_stream;
  const size_t need = c->lay.per_level * p->n_levels + c->lay.shared;
  if (arena) {
    if (arena_bytes < need || ((uintptr_t)arena & 255)) {
      delete c;
      return SACRA_ERR_OOM;
    }
    c->arena = (char *)arena;
  } else {
    if (cudaMalloc(&c->arena, need) != cudaSuccess) {
      cudaGetLastError();
      delete c;
      return SACRA_ERR_OOM;
    }
    c->own_arena = true;
  }
  if (cudaMemsetAsync(c->arena, 0, need, c->stream) != cudaSuccess) {
    cudaGetLastError();
    if (c->own_arena) cudaFree(c->arena);
    delete c;
    return SACRA_ERR_CUDA;
  }
  fill_dev_params(p, &c->dp);

  char *shared = c->arena + c->lay.per_level * p->n_levels;
  c->ds = (double *)(shared + c->lay.ds_off);
  double *dy = (double *)(shared + c->lay.dy_off);
  double *dyy = (double *)(shared + c->lay.dyy_off);
  c->tab = (double *)(shared + c->lay.tab_off);
  c->part = (double *)(shared + c->lay.part_off);
  c->dout = (double *)(shared + c->lay.dout_off);
  c->nfb = (unsigned long long *)(shared + c->lay.nfb_off);
  const size_t P = c->lay.P;
  const size_t rwp = round_up((size_t)c->lay.rw, 32);
  for (int l = 0; l < p->n_levels; ++l) {
    Lev &L = c->lv[l];
    char *b = c->arena + c->lay.per_level * l;
    L.nx = p->nx; L.nz = p->nz; L.px = p->nx + 2 * GH; L.pz = p->nz + 2 * GH; L.rw = (int)rwp;
    L.dx = p->dx0 / (double)(1 << l);
    L.dz = p->dz0 / (double)(1 << l);
    L.i60x = 1.0 / (60.0 * L.dx);
    L.i60z = 1.0 / (60.0 * L.dz);
    L.P = P;
    double *dp = (double *)b;
    L.un = dp; dp += NST * P;
    L.us = dp; dp += NST * P;
    L.ka = dp; dp += NST * P;
    L.rhs = dp; dp += NST * P;
    L.prim = dp; dp += NPRIM * P;
    L.fx = dp; dp += NCONS * P;
    L.fz = dp; dp += NCONS * P;
    L.freg = dp; dp += 4 * NCONS * rwp;
    L.status = (int *)dp;
    L.dy = dy; L.dyy = dyy;
    L.nfb = c->nfb;
  }
  // cartoon table: for x_j = (j - 1/2) dx and plane m dy (dy = dx), the
  // 9 weights on x_{j-4..j+4} at varpi = sqrt(x_j^2 + (m dy)^2), cos, sin of phi, cos - 1
  {
    const int nj = p->nx + 8;
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
    cudaMemcpyAsync(c->tab, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream);
  }
  {
    GridWeights w;
    double n8[8];
    for (int n = 0; n < 8; ++n) n8[n] = n - 3;
    lagrange_weights(8, n8, 0.25, w.prol);
    lagrange_weights(8, n8, 0.5, w.rest_c);          // nodes 2j-4..2j+3 relative to 2j-1
    for (int n = 0; n < 8; ++n) n8[n] = n;
    lagrange_weights(8, n8, 4.5, w.rest_s1);         // N-7..N -> N - 5/2
    lagrange_weights(8, n8, 6.5, w.rest_s0);         // N-7..N -> N - 1/2
    set_grid_weights(w);
  }
  if (cudaStreamSynchronize(c->stream) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
    if (c->own_arena) cudaFree(c->arena);
    delete c;
    return SACRA_ERR_CUDA;
  }
  *out = c;
  return SACRA_OK;
}

sacra_status sacra_set_initial_data(sacra_ctx *c, int level, int kind, const double *host, int n_fields) {
  if (!c) return SACRA_ERR_ARG;
  if (level < 0 || level >= c->prm.n_levels || !host) return fail(c, SACRA_ERR_ARG, "bad level or buffer");
  if (n_fields != 30) return fail(c, SACRA_ERR_ARG, "n_fields must be 30");
  Lev &L = c->lv[level];
  const size_t np = (size_t)L.px * L.pz;
  if (kind == SACRA_PRIM_METRIC) {
    for (int f = 0; f < NMET; ++f)
      cudaMemcpyAsync(L.un + (size_t)f * L.P, host + (size_t)f * np, np * 8, cudaMemcpyHostToDevice, c->stream);
    for (int v = 0; v < 5; ++v)
      cudaMemcpyAsync(L.prim + (size_t)v * L.P, host + (size_t)(NMET + v) * np, np * 8, cudaMemcpyHostToDevice,
                      c->stream);
    run(c, K_PRIM2CONS, (long long)np, [&] { launch_prim2cons_all(L, c->dp, L.un, c->stream); });
  } else if (kind == SACRA_RAW) {
    for (int f = 0; f < NST; ++f)
      cudaMemcpyAsync(L.un + (size_t)f * L.P, host + (size_t)f * np, np * 8, cudaMemcpyHostToDevice, c->stream);
    run(c, K_C2P, (long long)np, [&] { launch_c2p_region(L, c->dp, L.un, 1 - GH, L.nx + GH, 1 - GH, L.nz + GH, c->stream); });
  } else {
    return fail(c, SACRA_ERR_ARG, "unknown kind");
  }
  cudaMemcpyAsync(L.us, L.un, (size_t)NST * L.P * 8, cudaMemcpyDeviceToDevice, c->stream);
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return cuda_check(c, "set_initial_data");
  c->have_data[level] = true;
  return cuda_check(c, "set_initial_data");
}

static bool ready(sacra_ctx *c) {
  for (int l = 0; l < c->prm.n_levels; ++l)
    if (!c->have_data[l]) return false;
  return true;
}

sacra_status sacra_regrid_ghosts(sacra_ctx *c, int what, int stage, double dt) {
  if (!c) return SACRA_ERR_ARG;
  if (!ready(c)) return fail(c, SACRA_ERR_STATE, "initial data missing on some level");
  if (what == SACRA_FILL) {
    if (stage < 0 || stage >= n_stages(c)) return fail(c, SACRA_ERR_ARG, "bad stage");
    enqueue_fill(c, stage, dt);
  } else if (what == SACRA_RESTRICT_REFLUX) {
    enqueue_restrict(c);
  } else {
    return fail(c, SACRA_ERR_ARG, "unknown regrid request");
  }
  return cuda_check(c, "regrid_ghosts");
}

sacra_status sacra_rk_stage(sacra_ctx *c, int stage, double dt) {
  if (!c) return SACRA_ERR_ARG;
  if (!ready(c)) return fail(c, SACRA_ERR_STATE, "initial data missing on some level");
  if (stage < 0 || stage >= n_stages(c) || !(dt > 0)) return fail(c, SACRA_ERR_ARG, "bad stage or dt");
  enqueue_stage(c, stage, dt);
  return cuda_check(c, "rk_stage");
}

sacra_status sacra_step(sacra_ctx *c, double dt, int n_steps, int use_graph) {
  if (!c) return SACRA_ERR_ARG;
  if (!ready(c)) return fail(c, SACRA_ERR_STATE, "initial data missing on some level");
  if (!(dt > 0) || n_steps < 0) return fail(c, SACRA_ERR_ARG, "bad dt or n_steps");
  for (int it = 0; it < n_steps; ++it) {
    if (!use_graph) {
      enqueue_step(c, dt);
      continue;
    }
    const int par = c->parity;
    if (!c->gexec[par] || c->gdt[par] != dt) {
      if (c->gexec[par]) { cudaGraphExecDestroy(c->gexec[par]); c->gexec[par] = nullptr; }
      cudaGraph_t g;
      const long long before = c->launches;
      if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return cuda_check(c, "graph capture (the stream must be a non-default stream)");
      c->capturing = true;
      enqueue_step(c, dt);       // swaps the registers on the host side
      c->capturing = false;
      if (cudaStreamEndCapture(c->stream, &g) != cudaSuccess) return cuda_check(c, "graph capture");
      c->glaunch[par] = c->launches - before;
      c->launches = before;
      swap_registers(c);         // undo: the graph has not run yet
      if (cudaGraphInstantiate(&c->gexec[par], g, 0) != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_check(c, "graph instantiate");
      }
      cudaGraphDestroy(g);
      c->gdt[par] = dt;
    }
    if (cudaGraphLaunch(c->gexec[par], c->stream) != cudaSuccess) return cuda_check(c, "graph launch");
    c->launches += c->glaunch[par];
    c->dt_step = dt;
    swap_registers(c);
  }
  return cuda_check(c, "step");
}

sacra_status sacra_read_state(sacra_ctx *c, int level, int which, int field, double *host, size_t n) {
  if (!c) return SACRA_ERR_ARG;
  if (level < 0 || level >= c->prm.n_levels || !host) return fail(c, SACRA_ERR_ARG, "bad level or buffer");
  Lev &L = c->lv[level];
  const size_t np = (size_t)L.px * L.pz;
  const double *src = nullptr;
  std::vector<double> tmp;
  if (which == SACRA_STATE_STEP || which == SACRA_STATE_STAGE || which == SACRA_RHS) {
    if (field < 0 || field >= NST) return fail(c, SACRA_ERR_ARG, "bad field");
    const double *base = which == SACRA_STATE_STEP ? L.un : (which == SACRA_STATE_STAGE ? L.us : L.rhs);
    src = base + (size_t)field * L.P;
  } else if (which == SACRA_PRIMS) {
    if (field < 0 || field >= NPRIM) return fail(c, SACRA_ERR_ARG, "bad field");
    src = L.prim + (size_t)field * L.P;
  } else if (which != SACRA_STATUS) {
    return fail(c, SACRA_ERR_ARG, "unknown plane");
  }
  tmp.resize(np);
  if (which == SACRA_STATUS) {
    std::vector<int> st(np);
    cudaMemcpyAsync(st.data(), L.status, np * 4, cudaMemcpyDeviceToHost, c->stream);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return cuda_check(c, "read_state");
    for (size_t i = 0; i < np; ++i) tmp[i] = st[i];
  } else {
    cudaMemcpyAsync(tmp.data(), src, np * 8, cudaMemcpyDeviceToHost, c->stream);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return cuda_check(c, "read_state");
  }
  if (n == np) {
    memcpy(host, tmp.data(), np * 8);
  } else if (n == (size_t)L.nx * L.nz) {
    for (int k = 1; k <= L.nz; ++k) memcpy(host + (size_t)(k - 1) * L.nx, tmp.data() + cid(L, 1, k), (size_t)L.nx * 8);
  } else {
    return fail(c, SACRA_ERR_ARG, "n must be nx*nz or px*pz");
  }
  return cuda_check(c, "read_state");
}

sacra_status sacra_constraints(sacra_ctx *c, sacra_diag *out) {
  if (!c || !out) return SACRA_ERR_ARG;
  if (!ready(c)) return fail(c, SACRA_ERR_STATE, "initial data missing on some level");
  enqueue_fill(c, 0, 0.0);
  const int L = c->prm.n_levels;
  int slot = 0;
  for (int l = 0; l < L; ++l) {
    Lev &lv = c->lv[l];
    const long long cells = (long long)lv.nx * lv.nz;
    if (c->prm.evolve_spacetime) {
      run(c, K_CARTOON, (long long)(lv.nx + 7) * (lv.nz + 10), [&] { launch_cartoon(lv, c->dp, lv.un, c->tab, kTabStride, c->stream); });
      run(c, K_Z4C_DERIVS, cells, [&] { launch_z4c_derivs(lv, c->dp, lv.un, c->ds, lv.nx, lv.nz, c->stream); });
    }
    const int sl = slot;
    run(c, K_DIAG, cells, [&] { launch_diag(lv, c->dp, c->ds, l < L - 1, c->prm.evolve_spacetime, c->part, sl, c->stream); });
    slot += diag_blocks(lv);
  }
  run(c, K_DIAG_FINAL, slot, [&] { launch_diag_final(c->part, slot, c->dout, c->stream); });
  double h[9];
  unsigned long long nfb = 0;
  cudaMemcpyAsync(h, c->dout, sizeof(h), cudaMemcpyDeviceToHost, c->stream);
  cudaMemcpyAsync(&nfb, c->nfb, sizeof(nfb), cudaMemcpyDeviceToHost, c->stream);
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return cuda_check(c, "constraints");
  out->H_L2 = sqrt(h[0] / h[4]);
  for (int a = 0; a < 3; ++a) out->M_L2[a] = sqrt(h[1 + a] / h[4]);
  out->Mb = h[5];
  out->J = h[6];
  out->rho_max = h[7];
  out->n_c2p_fail = h[8];
  out->n_fallback = (double)nfb;
  return cuda_check(c, "constraints");
}

sacra_status sacra_sync(sacra_ctx *c) {
  if (!c) return SACRA_ERR_ARG;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return cuda_check(c, "sync");
  return cuda_check(c, "sync");
}

long long sacra_launch_count(const sacra_ctx *c) { return c ? c->launches : -1; }

sacra_status sacra_profile(sacra_ctx *c, int enable) {
  if (!c) return SACRA_ERR_ARG;
  c->prof = enable != 0;
  c->recs.clear();
  c->pool_used = 0;
  return SACRA_OK;
}

sacra_status sacra_profile_get(sacra_ctx *c, int idx, char *name, size_t name_len, double *total_ms,
                               long long *launches, long long *cells) {
  if (!c || idx < 0 || idx >= K_COUNT || !name || name_len == 0) return SACRA_ERR_ARG;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return cuda_check(c, "profile_get");
  double ms = 0.0;
  long long n = 0, cl = 0;
  for (const ProfRec &r : c->recs) {
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
  return cuda_check(c, "profile_get");
}

void sacra_destroy(sacra_ctx *c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  for (int i = 0; i < 2; ++i)
    if (c->gexec[i]) cudaGraphExecDestroy(c->gexec[i]);
  for (cudaEvent_t e : c->pool) cudaEventDestroy(e);
  if (c->own_arena) cudaFree(c->arena);
  delete c;
}

const char *sacra_last_error(const sacra_ctx *c) { return c ? c->err.c_str() : "null context"; }

}  // extern "C"
