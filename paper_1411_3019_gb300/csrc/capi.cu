// capi.cu -- the C ABI of include/md.h on top of the kernels of kernels.cu.
//
// A handle owns every device buffer it allocates (cudaMalloc in md_create,
// cudaFree in md_destroy). One md_step enqueues, per time step, the kernels
// pair -> integrate -> scan (3) -> scatter -> bucket build; the step is
// captured once into a CUDA graph (the step counter and the first-step flag
// live in device memory, so one graph serves every step) and replayed.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/md.h"
#include "engine.h"

using namespace surfmd;

constexpr uint32_t kDefaultSpinLimit = 1u << 22;  // reads of one scan word before the wait gives up

struct md_handle {
  int dev = 0;
  int fused_rebuild = 1;     // Verlet-list step: the cell-list and list rebuild as one cooperative launch
  int rebuild_ctas = 0;      // CTAs of that launch (0: not computed yet)
  bool cells_stale = false;  // a step's cell list was not completed (a bounded wait ran out)
  cudaStream_t user_stream = nullptr;  // set by md_set_stream (nullptr: own stream)
  cudaStream_t own_stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  int precision = 1;
  int64_t n = 0;
  int nsys = 0;
  int has_pairs = 0, bonds = 0, walls = 0, excl = 0, bends = 0;
  bool state_set = false;
  std::vector<SysDev> sys;
  std::vector<int64_t> first;
  TypeTable types{};
  DevArrays A{};
  int64_t* d_first = nullptr;
  double* d_stage = nullptr;   // 9n doubles
  int32_t* d_stage_i = nullptr;  // 2n int32 (type, mol)
  uint8_t* d_stage_u8 = nullptr; // n
  unsigned long long* d_resid = nullptr;
  double* d_obs = nullptr;
  uint32_t* h_status = nullptr;  // pinned
  unsigned long long* h_resid = nullptr;  // pinned
  cudaGraphExec_t graph = nullptr;
  // visiting order of the pair kernel (refreshed every kOrderEvery steps)
  DevArrays O{};
  uint32_t order_coord_shift = 0, order_morton_drop = 0, order_sys_shift = 0;
  uint32_t* d_order = nullptr;
  int64_t steps_since_order = 0;
  int64_t last_launches = 0;
  // Verlet neighbour list (md_set_neighbor_list); A.nl_dirty != null when on
  uint32_t* d_nl_dirty = nullptr;
  int32_t nl_capacity = 0;  // entries per particle the allocated list holds
  // resident engine (MD_OPT_ENGINE = 1): systems largest first, a work counter
  int engine = 0;
  int res_threads = 0;  // 0: chosen per size class
  int64_t res_steps_per_launch = 256;
  uint32_t res_nmax = 0, res_tmax = 0;
  int32_t* d_res_order = nullptr;
  uint32_t* d_res_next = nullptr;
  std::vector<int64_t> res_n_sorted;  // system sizes in work-list order (largest first)
  std::vector<uint32_t> res_t_sorted;  // their bucket counts
  struct ResClass {
    int32_t offset, count;
    uint32_t nmax, tmax;
    int threads;
  };
  std::vector<ResClass> res_classes;  // launches of one resident chunk
  std::vector<void*> allocs;
  std::string err;

  cudaStream_t stream() const { return user_stream ? user_stream : own_stream; }
};

static std::string g_create_err;
constexpr int64_t kOrderEvery = 16;  // steps between refreshes of the pair visiting order

namespace {

int fail(md_handle* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  else g_create_err = msg;
  return code;
}

int cuda_fail(md_handle* h, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  return fail(h, MD_ERR_CUDA, m);
}

#define CK(h, call)                                   \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
  } while (0)

template <typename T>
cudaError_t dalloc(md_handle* h, T** p, size_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
  if (e == cudaSuccess) {
    h->allocs.push_back(q);
    *p = static_cast<T*>(q);
  }
  return e;
}

// double-float copy of a float64 constant: h = v rounded to float32, l = the rest rounded
DF df_split(double v) {
  DF r;
  r.h = (float)v;
  r.l = (float)(v - (double)r.h);
  return r;
}

bool symmetric_ok(const double t[MD_MAX_TYPES][MD_MAX_TYPES], int nt) {
  for (int a = 0; a < nt; ++a)
    for (int b = 0; b < nt; ++b)
      if (!(t[a][b] == t[b][a]) || !std::isfinite(t[a][b]) || t[a][b] < 0.0) return false;
  return true;
}

// Validate one system's parameters and fill its SysDev (grid left to the caller).
int check_system(const md_surface& s, const md_params& p, SysDev& S, std::string& why) {
  auto bad = [&](const char* m) {
    why = m;
    return MD_ERR_INVALID_ARG;
  };
  if (!(p.dt > 0.0) || !std::isfinite(p.dt)) return bad("dt must be > 0");
  if (!(p.kT >= 0.0) || !(p.gamma >= 0.0)) return bad("kT and gamma must be >= 0");
  if (!(p.rattle_tol > 0.0)) return bad("rattle_tol must be > 0");
  if (p.max_newton < 0 || p.max_newton > 10000) return bad("max_newton out of range");
  if (p.precision != MD_PREC_FP64 && p.precision != MD_PREC_MIXED) return bad("unknown precision");
  if (p.ntypes < 1 || p.ntypes > MD_MAX_TYPES) return bad("ntypes must be in 1..8");
  for (int a = 0; a < p.ntypes; ++a)
    if (!(p.mass[a] > 0.0)) return bad("masses must be > 0");
  if (!symmetric_ok(p.eps, p.ntypes) || !symmetric_ok(p.sigma, p.ntypes) || !symmetric_ok(p.rcut, p.ntypes))
    return bad("eps, sigma and rcut must be symmetric, finite and >= 0");
  for (int a = 0; a < p.ntypes; ++a)
    for (int b = 0; b < p.ntypes; ++b)
      if (p.rcut[a][b] > 0.0 && !(p.sigma[a][b] > 0.0)) return bad("sigma must be > 0 where rcut > 0");
  if (s.kind < MD_SURF_NONE || s.kind > MD_SURF_THYLAKOID) return bad("unknown surface kind");
  if (s.reserved != 0) return bad("reserved fields must be 0");
  if (p.pair_form != MD_PAIR_TRUNC_SHIFT && p.pair_form != MD_PAIR_LINEAR_SMOOTH) return bad("unknown pair_form");
  for (int d = 0; d < 3; ++d)
    if (p.periodic[d] && !(p.box_hi[d] > p.box_lo[d])) return bad("a periodic axis needs box_hi > box_lo");
  if (p.beads_per_mol > 1 && !(p.bond_k >= 0.0 && p.bond_r0 >= 0.0)) return bad("bond_k, bond_r0 >= 0");
  if (p.wall_kind != MD_WALL_PLANES && p.wall_kind != MD_WALL_SPHERE) return bad("unknown wall_kind");
  if (p.wall_enable && p.wall_kind == MD_WALL_PLANES &&
      !(p.wall_hi_z > p.wall_lo_z && p.wall_sigma > 0.0 && p.wall_eps >= 0.0))
    return bad("wall needs wall_hi_z > wall_lo_z and wall_sigma > 0");
  if (p.wall_enable && p.wall_kind == MD_WALL_SPHERE &&
      !(p.wall_radius >= 0.0 && p.wall_sigma > 0.0 && p.wall_eps >= 0.0 && std::isfinite(p.wall_center[0]) &&
        std::isfinite(p.wall_center[1]) && std::isfinite(p.wall_center[2])))
    return bad("a spherical wall needs wall_radius >= 0, wall_sigma > 0 and a finite wall_center");
  if (!(p.angle_k >= 0.0 && std::isfinite(p.angle_k) && std::isfinite(p.angle_theta0)))
    return bad("angle_k must be >= 0 and finite");
  if (p.angle_k > 0.0 && p.beads_per_mol < 3) return bad("bend angles need beads_per_mol >= 3");
  if (p.bond_r0_mix != 0 && p.bond_r0_mix != 1) return bad("bond_r0_mix must be 0 or 1");
  std::memset(&S, 0, sizeof(S));
  S.kind = s.kind;
  for (int d = 0; d < 3; ++d) S.c[d] = s.center[d];
  for (int d = 0; d < 4; ++d) S.p[d] = s.p[d];
  switch (s.kind) {
    case MD_SURF_PLANE:
      if (!(s.p[0] * s.p[0] + s.p[1] * s.p[1] + s.p[2] * s.p[2] > 0.0)) return bad("plane normal is zero");
      break;
    case MD_SURF_SPHERE:
      if (!(s.p[0] > 0.0)) return bad("sphere radius must be > 0");
      break;
    case MD_SURF_ELLIPSOID:
      for (int d = 0; d < 3; ++d) {
        if (!(s.p[d] > 0.0)) return bad("ellipsoid semi-axes must be > 0");
        S.inv_a2[d] = 1.0 / (s.p[d] * s.p[d]);
      }
      break;
    case MD_SURF_TORUS:
      if (!(s.p[0] > s.p[1] && s.p[1] > 0.0)) return bad("torus needs R > r > 0");
      break;
    case MD_SURF_GAUSSIAN_BUMP:
      if (!(s.p[1] > 0.0)) return bad("bump width must be > 0");
      if (!p.periodic[0] || !p.periodic[1]) return bad("the bump needs periodic x and y");
      break;
    case MD_SURF_XY2D:
      if (!p.periodic[0] || !p.periodic[1] || p.periodic[2])
        return bad("the 2D plane needs periodic x and y and an open z axis");
      break;
    case MD_SURF_THYLAKOID:
      if (!(s.p[0] > 0.0 && s.p[1] > 0.0 && s.p[2] > 0.0 && s.p[3] > 0.0))
        return bad("the thylakoid needs R_b, L_x, R_c, L_b > 0");
      if (p.periodic[0] || p.periodic[1] || !p.periodic[2]) return bad("the thylakoid needs periodic z and open x, y");
      break;
    case MD_SURF_CYLINDER:
      if (!(s.p[0] > 0.0)) return bad("cylinder radius must be > 0");
      if (!(s.p[1] == 0.0 || s.p[1] == 1.0 || s.p[1] == 2.0)) return bad("cylinder axis must be 0, 1 or 2");
      S.axis = (int)s.p[1];
      break;
    default:
      break;
  }
  for (int d = 0; d < 3; ++d) {
    S.c_f[d] = (float)S.c[d];
    S.inv_a2_f[d] = (float)S.inv_a2[d];
  }
  for (int d = 0; d < 4; ++d) S.p_f[d] = (float)S.p[d];
  S.dt = p.dt;
  S.half_dt = 0.5 * p.dt;
  S.kT = p.kT;
  S.gamma = p.gamma;
  S.comb = 1.0 / (1.0 + 0.5 * p.gamma * p.dt);
  S.noise_unit = std::sqrt(2.0 * p.kT * p.gamma / p.dt);
  S.tol = p.rattle_tol;
  S.tol2 = p.rattle_tol * p.rattle_tol;
  S.gamma_f = (float)p.gamma;
  S.comb_f = (float)S.comb;
  S.noise_unit_f = (float)S.noise_unit;
  S.max_newton = p.max_newton;
  S.frozen = p.frozen_normal ? 1 : 0;
  for (int t = 0; t < kMaxTypes; ++t) {
    if (!(p.mass[t] > 0.0)) continue;
    S.dtm[t] = p.dt / p.mass[t];
    S.inv_dtm[t] = p.mass[t] / p.dt;
    S.dtm_f[t] = (float)S.dtm[t];
  }
  S.half_dt_f = (float)S.half_dt;
  S.tol_f = (float)p.rattle_tol;
  if (s.kind == MD_SURF_SPHERE || s.kind == MD_SURF_CYLINDER) S.gconst = -s.p[0] * s.p[0];
  if (s.kind == MD_SURF_TORUS) S.gconst = -s.p[1] * s.p[1];
  S.c_zero = (S.c[0] == 0.0 && S.c[1] == 0.0 && S.c[2] == 0.0) ? 1 : 0;
  for (int d = 0; d < 3; ++d) {
    S.c_df[d] = df_split(S.c[d]);
    S.inv_a2_df[d] = df_split(S.inv_a2[d]);
    S.pn_df[d] = df_split(s.kind == MD_SURF_PLANE ? s.p[d] : 0.0);
  }
  S.gconst_df = df_split(S.gconst);
  S.R_df = df_split(s.kind == MD_SURF_TORUS ? s.p[0] : 0.0);
  S.dt_df = df_split(S.dt);
  S.half_dt_df = df_split(S.half_dt);
  for (int t = 0; t < kMaxTypes; ++t) {
    S.dtm_df[t] = df_split(S.dtm[t]);
    S.inv_dtm_df[t] = df_split(S.inv_dtm[t]);
  }
  for (int d = 0; d < 3; ++d) {
    S.box_lo[d] = p.box_lo[d];
    S.box_len[d] = p.box_hi[d] - p.box_lo[d];
    S.inv_box_len[d] = S.box_len[d] > 0.0 ? 1.0 / S.box_len[d] : 0.0;
    S.periodic[d] = p.periodic[d] ? 1 : 0;
  }
  S.bpm = p.beads_per_mol;
  S.excl = p.exclude_intramol ? 1 : 0;
  S.bond_k = p.bond_k;
  S.bond_r0 = p.bond_r0;
  S.wall = p.wall_enable ? 1 : 0;
  S.wall_lo = p.wall_lo_z;
  S.wall_hi = p.wall_hi_z;
  S.wall_eps = p.wall_eps;
  S.angle_k = p.angle_k;
  S.angle_theta0 = p.angle_theta0;
  S.angle_sin0 = std::sin(p.angle_theta0);
  S.angle_cos0 = std::cos(p.angle_theta0);
  S.bond_mix = p.bond_r0_mix;
  S.wall_kind = p.wall_kind;
  S.wall_radius = p.wall_radius;
  for (int d = 0; d < 3; ++d) S.wall_center[d] = p.wall_center[d];
  S.wall_sigma = p.wall_sigma;
  S.wall_rc = std::pow(2.0, 1.0 / 6.0) * p.wall_sigma;
  S.seed_lo = (uint32_t)(p.seed & 0xffffffffu);
  S.replica = p.replica;
  return MD_OK;
}

// Extent of the surface along axis d: returns false if unbounded.
bool surface_extent(const md_surface& s, int d, double& lo, double& hi) {
  const double c = s.center[d];
  switch (s.kind) {
    case MD_SURF_SPHERE: lo = c - s.p[0]; hi = c + s.p[0]; return true;
    case MD_SURF_ELLIPSOID: lo = c - s.p[d]; hi = c + s.p[d]; return true;
    case MD_SURF_TORUS: {
      const double e = (d < 2) ? s.p[0] + s.p[1] : s.p[1];
      lo = c - e; hi = c + e;
      return true;
    }
    case MD_SURF_XY2D:
      if (d < 2) return false;
      lo = c; hi = c;
      return true;
    case MD_SURF_THYLAKOID: {
      if (d == 2) return false;
      const double w = s.p[1] + 2.0 * s.p[2];  // block width
      const double e = d == 0 ? 0.5 * s.p[3] + s.p[2] + w : 0.5 * w;
      lo = c - e; hi = c + e;
      return true;
    }
    case MD_SURF_CYLINDER:
      if (d == (int)s.p[1]) return false;
      lo = c - s.p[0]; hi = c + s.p[0];
      return true;
    case MD_SURF_GAUSSIAN_BUMP:
      if (d < 2) return false;
      lo = c + std::min(0.0, s.p[0]); hi = c + std::max(0.0, s.p[0]);
      return true;
    case MD_SURF_PLANE: {
      const int o1 = (d + 1) % 3, o2 = (d + 2) % 3;
      if (s.p[o1] == 0.0 && s.p[o2] == 0.0) {
        lo = hi = c;
        return true;
      }
      return false;
    }
    default:
      return false;
  }
}

void fill_types(const md_params& p, TypeTable& T) {
  std::memset(&T, 0, sizeof(T));
  for (int a = 0; a < kMaxTypes; ++a) {
    const double m = a < p.ntypes ? p.mass[a] : 1.0;
    T.mass[a] = m;
    T.inv_mass[a] = 1.0 / m;
    T.sqrt_mass[a] = std::sqrt(m);
    T.sqrt_mass_f[a] = (float)std::sqrt(m);
    for (int b = 0; b < kMaxTypes; ++b) {
      if (a >= p.ntypes || b >= p.ntypes) continue;
      const double rc = p.rcut[a][b], sg = p.sigma[a][b], ep = p.eps[a][b];
      T.eps[a][b] = ep;
      T.sig2[a][b] = sg * sg;
      T.rc2[a][b] = rc * rc;
      double shift = 0.0;
      if (rc > 0.0) {
        const double s6 = std::pow(sg / rc, 6.0);
        shift = 4.0 * ep * (s6 * s6 - s6);
      }
      T.shift[a][b] = shift;
      // linear smoothing: phi'(r_c) (0 for the truncated-shifted form)
      double lin = 0.0;
      if (rc > 0.0 && p.pair_form == MD_PAIR_LINEAR_SMOOTH) {
        const double s6 = std::pow(sg / rc, 6.0);
        lin = -24.0 * ep * (2.0 * s6 * s6 - s6) / rc;
      }
      T.lin[a][b] = lin;
      T.rc[a][b] = rc;
      T.bond_r0_mix[a][b] = std::pow(2.0, 1.0 / 6.0) * sg / 2.0;
      T.eps_f[a][b] = (float)ep;
      T.sig2_f[a][b] = (float)(sg * sg);
      T.rc2_f[a][b] = (float)(rc * rc);
      T.shift_f[a][b] = (float)shift;
      T.lin_f[a][b] = (float)lin;
      T.rc_f[a][b] = (float)rc;
      // mixed path, pair terms from double-float displacements
      const double sg6 = std::pow(sg * sg, 3.0);
      T.rc2m_f[a][b] = (float)(rc * rc * (1.0 + std::ldexp(1.0, -18)));
      T.rc2_df[a][b] = df_split(rc * rc);
      T.s6x2_df[a][b] = df_split(2.0 * sg6);
      T.c24_f[a][b] = (float)(24.0 * ep * sg6);
      T.c4_f[a][b] = (float)(4.0 * ep * sg6);
      T.s6_f[a][b] = (float)sg6;
    }
  }
}

bool same_interactions(const md_params& a, const md_params& b) {
  if (a.precision != b.precision || a.ntypes != b.ntypes || a.cell_size != b.cell_size ||
      a.pair_form != b.pair_form)
    return false;
  for (int i = 0; i < a.ntypes; ++i) {
    if (a.mass[i] != b.mass[i]) return false;
    for (int j = 0; j < a.ntypes; ++j)
      if (a.eps[i][j] != b.eps[i][j] || a.sigma[i][j] != b.sigma[i][j] || a.rcut[i][j] != b.rcut[i][j])
        return false;
  }
  return true;
}

int check_device_status(md_handle* h) {
  CK(h, cudaMemcpyAsync(h->h_status, h->A.status, sizeof(uint32_t), cudaMemcpyDeviceToHost, h->stream()));
  CK(h, cudaStreamSynchronize(h->stream()));
  const uint32_t st = *h->h_status;
  if (st == 0) return MD_OK;
  CK(h, cudaMemsetAsync(h->A.status, 0, sizeof(uint32_t), h->stream()));
  CK(h, cudaStreamSynchronize(h->stream()));
  if (st & kFlagRattle) return fail(h, MD_ERR_RATTLE_DIVERGED, "RATTLE Newton iteration missed the tolerance");
  if (st & kFlagNonfinite) return fail(h, MD_ERR_NONFINITE, "non-finite position or momentum");
  if (st & kFlagOutOfGrid) return fail(h, MD_ERR_OUT_OF_GRID, "a particle left its cell grid or crossed a wall");
  if (st & kFlagTimeout) {  // the cell list of that step is not valid: rebuild it before the next step
    h->cells_stale = true;
    return fail(h, MD_ERR_TIMEOUT, "a bounded device wait ran out (the cell list is rebuilt before the next step)");
  }
  if (st & kFlagNlistFull)
    return fail(h, MD_ERR_NLIST_FULL, "a particle has more neighbours than the neighbour list holds");
  if (st & kFlagOffSurface)
    return fail(h, MD_ERR_INVALID_ARG, "a constrained particle is off its surface, or bad input values");
  return MD_OK;
}

// Cell list of the current positions (no step advance).
int rebuild_cells(md_handle* h) {
  if (!h->has_pairs) return MD_OK;
  // the fused rebuild's grid barrier starts from zero (a timed-out launch may have left arrivals)
  CK(h, cudaMemsetAsync(h->A.gbar, 0, sizeof(GridBar), h->stream()));
  if (h->A.nl_dirty) {  // neighbour-list mode: raise the flag so every rebuild kernel runs
    const uint32_t one = 1u;
    CK(h, cudaMemcpyAsync(h->A.nl_dirty, &one, sizeof(one), cudaMemcpyHostToDevice, h->stream()));
  }
  CK(h, launch_bin(h->A, h->precision, h->stream()));
  CK(h, launch_cells_after_bin(h->A, 0, h->stream()));
  CK(h, launch_bucket_build(h->A, h->precision, h->stream()));
  if (h->A.nl_dirty) CK(h, launch_nl_build(h->A, h->precision, h->excl, h->stream()));
  CK(h, launch_order(h->A, h->O, h->order_coord_shift, h->order_morton_drop, h->order_sys_shift, h->d_order,
                     h->stream()));
  h->steps_since_order = 0;
  return MD_OK;
}

// The kernels of one time step, in launch order.
struct StepKernel {
  const char* name;
  cudaError_t (*fn)(md_handle*, cudaStream_t);
};

cudaError_t k_pair_step(md_handle* h, cudaStream_t st) {
  return launch_pair(h->A, h->precision, h->has_pairs, h->bonds, h->walls, h->excl, st);
}
cudaError_t k_bend_step(md_handle* h, cudaStream_t st) { return launch_bend(h->A, h->precision, st); }
cudaError_t k_integrate_step(md_handle* h, cudaStream_t st) {
  return launch_integrate(h->A, h->precision, h->has_pairs, st);
}
cudaError_t k_scan_step(md_handle* h, cudaStream_t st) { return launch_scan(h->A, 1, st); }
cudaError_t k_scatter_step(md_handle* h, cudaStream_t st) { return launch_scatter(h->A, st); }
cudaError_t k_bucket_step(md_handle* h, cudaStream_t st) {
  return launch_bucket_build(h->A, h->precision, st);
}
cudaError_t k_advance_step(md_handle* h, cudaStream_t st) { return launch_advance(h->A, st); }
cudaError_t k_bin_step(md_handle* h, cudaStream_t st) { return launch_bin(h->A, h->precision, st); }
cudaError_t k_nl_build_step(md_handle* h, cudaStream_t st) {
  return launch_nl_build(h->A, h->precision, h->excl, st);
}

const StepKernel kStepWithCells[] = {{"pair", k_pair_step},
                                     {"integrate", k_integrate_step},
                                     {"scan", k_scan_step},
                                     {"scatter", k_scatter_step},
                                     {"bucket_build", k_bucket_step}};
const StepKernel kStepWithCellsBends[] = {{"pair", k_pair_step},
                                          {"bend", k_bend_step},
                                          {"integrate", k_integrate_step},
                                          {"scan", k_scan_step},
                                          {"scatter", k_scatter_step},
                                          {"bucket_build", k_bucket_step}};
const StepKernel kStepNoCells[] = {{"pair", k_pair_step}, {"integrate", k_integrate_step},
                                   {"advance", k_advance_step}};
const StepKernel kStepNoCellsBends[] = {{"pair", k_pair_step}, {"bend", k_bend_step},
                                        {"integrate", k_integrate_step}, {"advance", k_advance_step}};

// Neighbour-list mode: the cell-list kernels and the list build return at
// once unless the integrator raised the rebuild flag (the scan still
// advances the step counter).
const StepKernel kStepNl[] = {{"pair", k_pair_step},       {"integrate", k_integrate_step},
                              {"bin", k_bin_step},         {"scan", k_scan_step},
                              {"scatter", k_scatter_step}, {"bucket_build", k_bucket_step},
                              {"nl_build", k_nl_build_step}};
cudaError_t k_rebuild_step(md_handle* h, cudaStream_t st) {
  return launch_rebuild(h->A, h->precision, h->excl, h->rebuild_ctas, st);
}
const StepKernel kStepNlFused[] = {{"pair", k_pair_step}, {"integrate", k_integrate_step}, {"rebuild", k_rebuild_step}};
const StepKernel kStepNlFusedBends[] = {
    {"pair", k_pair_step}, {"bend", k_bend_step}, {"integrate", k_integrate_step}, {"rebuild", k_rebuild_step}};
const StepKernel kStepNlBends[] = {{"pair", k_pair_step},       {"bend", k_bend_step},
                                   {"integrate", k_integrate_step}, {"bin", k_bin_step},
                                   {"scan", k_scan_step},       {"scatter", k_scatter_step},
                                   {"bucket_build", k_bucket_step}, {"nl_build", k_nl_build_step}};

int step_kernels(const md_handle* h, const StepKernel** list) {
  if (h->has_pairs && h->A.nl_dirty && h->fused_rebuild && h->rebuild_ctas > 0) {
    *list = h->bends ? kStepNlFusedBends : kStepNlFused;
    return h->bends ? 4 : 3;
  }
  if (h->has_pairs && h->A.nl_dirty) {
    *list = h->bends ? kStepNlBends : kStepNl;
    return h->bends ? 8 : 7;
  }
  if (h->has_pairs) {
    *list = h->bends ? kStepWithCellsBends : kStepWithCells;
    return h->bends ? 6 : 5;
  }
  *list = h->bends ? kStepNoCellsBends : kStepNoCells;
  return h->bends ? 4 : 3;
}

// One time step, enqueued on stream st.
cudaError_t enqueue_step(md_handle* h, cudaStream_t st) {
  const StepKernel* ks;
  const int nk = step_kernels(h, &ks);
  for (int i = 0; i < nk; ++i) {
    cudaError_t e = ks[i].fn(h, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int build_graph(md_handle* h) {
  if (h->graph) return MD_OK;
  if (h->has_pairs && h->A.nl_dirty && h->fused_rebuild && h->rebuild_ctas == 0) {
    h->rebuild_ctas = rebuild_blocks(h->precision, h->excl, h->n);
    if (h->rebuild_ctas <= 0) h->fused_rebuild = 0;  // not launchable here: five separate launches
  }
  cudaGraph_t g = nullptr;
  CK(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = enqueue_step(h, h->cap_stream);
  cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &g);
  if (e == cudaSuccess && e2 == cudaSuccess) {
    e = cudaGraphInstantiate(&h->graph, g, 0);
    cudaGraphDestroy(g);
  } else if (g) {
    cudaGraphDestroy(g);
  }
  const cudaError_t failed = e != cudaSuccess ? e : e2;
  if (failed != cudaSuccess && h->A.nl_dirty && h->fused_rebuild) {
    // a cooperative launch that cannot be captured here: the separate rebuild kernels instead
    cudaGetLastError();
    h->graph = nullptr;
    h->fused_rebuild = 0;
    return build_graph(h);
  }
  if (e2 != cudaSuccess) return cuda_fail(h, e2, "capture of one step");
  if (e != cudaSuccess) return cuda_fail(h, e, "capture or instantiation of one step");
  return MD_OK;
}

// The largest bucket count a system of n particles can have on the resident
// engine (2^k >= 2n, at least 64).
uint32_t res_t_bound(int64_t n) {
  uint32_t t = 64;
  while ((int64_t)t < 2 * n && t < (1u << 16)) t <<= 1;
  return t;
}

// Size classes of the resident engine: consecutive runs of the work list
// (largest systems first). A class's shared memory is sized for its largest
// system; its CTA size maximises the warps resident per SM (registers and
// shared memory both limit the CTAs), or is the fixed size `threads` (> 0).
// A class ends where a smaller system would fit more CTAs of that size.
// Returns "" or why the engine cannot run this handle.
std::string plan_resident(md_handle* h, int threads) {
  h->res_classes.clear();
  if (!h->has_pairs) return "the resident engine needs pair interactions";
  if (h->res_nmax > 65535) return "the resident engine holds at most 65535 particles per system";
  if (h->res_nmax == 0) return "the batch has no particles";
  const int cands_auto[] = {512, 384, 256, 128};
  std::vector<int> cands;
  if (threads > 0) cands.push_back(threads);
  else cands.assign(std::begin(cands_auto), std::end(cands_auto));
  auto ctas = [&](int64_t n, uint32_t t_b, int thr) {
    return resident_blocks_per_sm(h->precision, h->bonds, h->walls, h->excl, (uint32_t)n, t_b, thr);
  };
  const int nsys = (int)h->res_n_sorted.size();
  for (int i = 0; i < nsys;) {
    const int64_t nmax = h->res_n_sorted[(size_t)i];
    int best_t = 0, best_k = 0, best_w = 0;
    for (int thr : cands) {
      const int k = ctas(nmax, res_t_bound(nmax), thr);
      const int w = k * thr / 32;
      if (w > best_w || (w == best_w && w > 0 && thr > best_t)) {
        best_t = thr;
        best_k = k;
        best_w = w;
      }
    }
    if (best_w == 0)
      return "the largest system (" + std::to_string(nmax) + " particles, " +
             std::to_string(resident_smem_bytes(h->precision, (uint32_t)nmax, res_t_bound(nmax))) +
             " bytes of shared memory) does not fit one CTA" +
             (threads > 0 ? " of " + std::to_string(threads) + " threads" : std::string());
    uint32_t tmax = h->res_t_sorted[(size_t)i];
    int j = i + 1;
    while (j < nsys) {
      const int64_t nj = h->res_n_sorted[(size_t)j];
      if (nj > 0 && ctas(nj, res_t_bound(nj), best_t) > best_k) break;
      tmax = std::max(tmax, h->res_t_sorted[(size_t)j]);
      ++j;
    }
    h->res_classes.push_back({i, j - i, (uint32_t)std::max<int64_t>(nmax, 1), tmax, best_t});
    i = j;
  }
  return "";
}

constexpr int64_t kRebuildLaunches = 7;  // bin, scan, scatter, bucket build, visiting order (3)

// Enqueue nsteps steps of every system on the resident engine: chunks of at
// most res_steps_per_launch steps, one launch per size class per chunk, the
// step counter advanced after each chunk. Returns the launches.
cudaError_t enqueue_resident(md_handle* h, int64_t nsteps, cudaStream_t st, int64_t* launches) {
  for (int64_t done = 0; done < nsteps;) {
    const int64_t chunk = std::min(nsteps - done, h->res_steps_per_launch);
    for (const auto& c : h->res_classes) {
      ResidentJob J{h->d_res_order + c.offset, h->d_res_next, c.count, (int32_t)chunk, c.nmax, c.tmax};
      cudaError_t e = launch_resident(h->A, h->precision, J, h->bonds, h->walls, h->excl, c.threads, 0, st);
      if (e != cudaSuccess) return e;
      ++*launches;
    }
    cudaError_t e = launch_advance_n(h->A, (int32_t)chunk, st);
    if (e != cudaSuccess) return e;
    ++*launches;
    done += chunk;
  }
  return cudaSuccess;
}

// nsteps steps by the resident engine, then the global cell list of the new
// positions (read by md_forces, md_get_state, the global engine and the
// observables).
int resident_steps(md_handle* h, int64_t nsteps) {
  int64_t launches = 0;
  CK(h, enqueue_resident(h, nsteps, h->stream(), &launches));
  int rc = rebuild_cells(h);
  if (rc) return rc;
  h->last_launches = launches + kRebuildLaunches;
  return MD_OK;
}

int forces_now(md_handle* h) {
  CK(h, launch_pair(h->A, h->precision, h->has_pairs, h->bonds, h->walls, h->excl, h->stream()));
  if (h->bends) CK(h, launch_bend(h->A, h->precision, h->stream()));
  return MD_OK;
}

int momenta_now(md_handle* h) {
  int rc = forces_now(h);
  if (rc) return rc;
  CK(h, launch_finish(h->A, h->precision, h->stream()));
  return MD_OK;
}

int require_state(md_handle* h) {
  if (!h) return MD_ERR_INVALID_ARG;
  if (!h->state_set) return fail(h, MD_ERR_INVALID_ARG, "no state: call md_set_state first");
  if (cudaSetDevice(h->dev) != cudaSuccess) return fail(h, MD_ERR_CUDA, "cudaSetDevice failed");
  return MD_OK;
}

}  // namespace

extern "C" {

int md_version(void) { return (1 << 16) | 0; }

int md_create(const md_surface* surf, const md_params* prm, int64_t n, md_handle** out) {
  if (!surf || !prm) return fail(nullptr, MD_ERR_INVALID_ARG, "surf and prm must not be NULL");
  return md_create_batch(1, surf, prm, &n, out);
}

int md_create_batch(int32_t nsys, const md_surface* surfs, const md_params* prms, const int64_t* n_per_sys,
                    md_handle** out) {
  if (!out) return fail(nullptr, MD_ERR_INVALID_ARG, "out must not be NULL");
  *out = nullptr;
  if (nsys < 1 || !surfs || !prms || !n_per_sys) return fail(nullptr, MD_ERR_INVALID_ARG, "bad batch arguments");
  if (nsys > (1 << 27)) return fail(nullptr, MD_ERR_INVALID_ARG, "too many systems");
  md_handle* h = new md_handle();
  std::string why;
  int64_t total = 0;
  h->sys.resize(nsys);
  h->first.resize(nsys);
  for (int s = 0; s < nsys; ++s) {
    if (n_per_sys[s] < 0) {
      delete h;
      return fail(nullptr, MD_ERR_INVALID_ARG, "n must be >= 0");
    }
    if (check_system(surfs[s], prms[s], h->sys[s], why) != MD_OK) {
      delete h;
      return fail(nullptr, MD_ERR_INVALID_ARG, "system " + std::to_string(s) + ": " + why);
    }
    if (!same_interactions(prms[0], prms[s])) {
      delete h;
      return fail(nullptr, MD_ERR_INVALID_ARG,
                  "systems of a batch must share precision, ntypes, mass, eps, sigma, rcut, pair_form, cell_size");
    }
    h->first[s] = total;
    h->sys[s].first = total;
    h->sys[s].n = n_per_sys[s];
    total += n_per_sys[s];
  }
  if (total >= (int64_t(1) << 31)) {
    delete h;
    return fail(nullptr, MD_ERR_INVALID_ARG, "at most 2^31 - 1 particles");
  }
  const md_params& P0 = prms[0];
  h->n = total;
  h->nsys = nsys;
  h->precision = P0.precision;
  fill_types(P0, h->types);
  double rcmax = 0.0;
  for (int a = 0; a < P0.ntypes; ++a)
    for (int b = 0; b < P0.ntypes; ++b) rcmax = std::max(rcmax, P0.rcut[a][b]);
  h->has_pairs = rcmax > 0.0;
  for (int s = 0; s < nsys; ++s) {
    if (prms[s].beads_per_mol > 1) h->bonds = 1;
    if (prms[s].wall_enable) h->walls = 1;
    if (prms[s].exclude_intramol) h->excl = 1;
    if (prms[s].beads_per_mol > 2 && prms[s].angle_k != 0.0) h->bends = 1;
  }
  // cell grids
  // cell edge: the largest cutoff plus a 2^-12 margin, rounded up to a float
  // so that the stencil shift is exact in the float32 pair kernel
  const double rc_eff = (double)std::nextafter((float)(std::max(rcmax, P0.cell_size) * (1.0 + 1.0 / 4096.0)),
                                               INFINITY);
  uint64_t cell_total = 0;
  for (int s = 0; s < nsys; ++s) {
    SysDev& S = h->sys[s];
    const md_params& p = prms[s];
    for (int d = 0; d < 3; ++d) {
      if (!h->has_pairs) {
        S.nc[d] = 1;
        S.cs[d] = 1.0;
        S.grid_lo[d] = 0.0;
      } else if (surfs[s].kind == MD_SURF_XY2D && d == 2) {  // one layer of cells about z = c_z
        S.nc[d] = 1;
        S.cs[d] = rc_eff;
        S.grid_lo[d] = surfs[s].center[2] - 0.5 * rc_eff;
      } else if (p.periodic[d]) {
        const double L = p.box_hi[d] - p.box_lo[d];
        const int nc = (int)std::floor(L / rc_eff);
        if (nc < 3) {
          delete h;
          return fail(nullptr, MD_ERR_INVALID_ARG, "a periodic axis must be at least 3 cells long");
        }
        S.nc[d] = nc;
        S.cs[d] = L / nc;
        S.grid_lo[d] = p.box_lo[d];
      } else {
        double lo, hi;
        if (p.box_hi[d] > p.box_lo[d]) {
          lo = p.box_lo[d];
          hi = p.box_hi[d];
        } else if (surface_extent(surfs[s], d, lo, hi)) {
          lo -= 2.0 * rc_eff;
          hi += 2.0 * rc_eff;
        } else {
          delete h;
          return fail(nullptr, MD_ERR_INVALID_ARG,
                      "system " + std::to_string(s) + ": give box_lo/box_hi for an axis the surface does not bound");
        }
        const double span = hi - lo;
        const double ncd = std::ceil(span / rc_eff);
        if (ncd > 1e6) {
          delete h;
          return fail(nullptr, MD_ERR_INVALID_ARG, "cell grid too large along one axis");
        }
        S.nc[d] = std::max(1, (int)ncd);
        S.cs[d] = rc_eff;
        S.grid_lo[d] = lo;
      }
      S.inv_cs[d] = 1.0 / S.cs[d];
      S.cs_f[d] = (float)S.cs[d];
      S.grid_lo_f[d] = (float)S.grid_lo[d];
      S.inv_cs_f[d] = (float)S.inv_cs[d];
      S.box_lo_f[d] = (float)S.box_lo[d];
      S.box_len_f[d] = (float)S.box_len[d];
    }
    // Stencil pruning for surface-bound particles: a neighbour within rc on a
    // surface of curvature <= kappa lies within rc^2 kappa / 2 of the
    // particle's tangent plane; the slab is taken twice that plus 1e-3.
    {
      const md_surface& sf = surfs[s];
      double kappa = -1.0;
      switch (sf.kind) {
        case MD_SURF_PLANE: kappa = 0.0; break;
        case MD_SURF_SPHERE: kappa = 1.0 / sf.p[0]; break;
        case MD_SURF_CYLINDER: kappa = 1.0 / sf.p[0]; break;
        case MD_SURF_ELLIPSOID: {
          const double amax = std::max(sf.p[0], std::max(sf.p[1], sf.p[2]));
          const double amin = std::min(sf.p[0], std::min(sf.p[1], sf.p[2]));
          kappa = amax / (amin * amin);
          break;
        }
        case MD_SURF_TORUS: kappa = 1.0 / sf.p[1] + 1.0 / (sf.p[0] - sf.p[1]); break;
        case MD_SURF_GAUSSIAN_BUMP: kappa = 2.0 * std::fabs(sf.p[0]) / (sf.p[1] * sf.p[1]); break;
        case MD_SURF_THYLAKOID: kappa = std::max(1.0 / sf.p[0], 1.0 / sf.p[2]); break;
        default: break;
      }
      S.slab = (h->has_pairs && kappa >= 0.0 && rcmax * kappa < 0.5) ? (float)(rcmax * rcmax * kappa + 1e-3) : 0.0f;
    }
    S.cell_base = (uint32_t)cell_total;
    cell_total += (uint64_t)S.nc[0] * (uint64_t)S.nc[1] * (uint64_t)S.nc[2];
    if (cell_total >= 0xFFFFFFF0ull) {
      delete h;
      return fail(nullptr, MD_ERR_INVALID_ARG, "more than 2^32 cells in the batch");
    }
  }
  // resident engine: per-system buckets in shared memory, the local cell id
  // when the system's grid has at most 2^k >= 2n (and >= 64) cells, else a
  // hash table of 2^k buckets
  for (int s = 0; s < nsys; ++s) {
    SysDev& S = h->sys[s];
    uint32_t t = 64;
    int lg = 6;
    while ((int64_t)t < 2 * n_per_sys[s] && lg < 16) {
      t <<= 1;
      ++lg;
    }
    const uint64_t cells = (uint64_t)S.nc[0] * (uint64_t)S.nc[1] * (uint64_t)S.nc[2];
    if (cells <= t) {
      S.res_t = (uint32_t)cells;
      S.res_hashed = 0;
      S.res_log_t = 0;
    } else {
      S.res_t = t;
      S.res_hashed = 1;
      S.res_log_t = lg;
    }
    h->res_nmax = std::max<uint32_t>(h->res_nmax, (uint32_t)std::min<int64_t>(n_per_sys[s], 0xFFFFFFFF));
    h->res_tmax = std::max(h->res_tmax, S.res_t);
  }
  // buckets: the cell id itself when the grid is small, else a hash table of 2^k >= 4n buckets
  uint64_t t_hash = 16;
  int log_t = 4;
  while (t_hash < (uint64_t)std::max<int64_t>(4 * total, 16) && log_t < 30) {
    t_hash <<= 1;
    ++log_t;
  }
  DevArrays& A = h->A;
  A.n = total;
  A.nsys = nsys;
  if (h->has_pairs && cell_total <= std::max<uint64_t>(t_hash, uint64_t(1) << 20)) {
    A.hashed = 0;
    A.nbucket = (uint32_t)cell_total;
    A.log_t = 0;
  } else {
    A.hashed = 1;
    A.nbucket = (uint32_t)t_hash;
    A.log_t = log_t;
  }
  if (!h->has_pairs) A.nbucket = 1;
  A.pair_lanes = 1;
  A.pair_queue = 1;
  A.list_warp = 32;
  A.store_noise = 1;
  A.ntypes = prms[0].ntypes;
  A.spin_limit = kDefaultSpinLimit;
  A.rec_cell = (!h->excl && cell_total < (uint64_t(1) << 29)) ? 1 : 0;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    delete h;
    return fail(nullptr, MD_ERR_NO_DEVICE, "no CUDA device is visible");
  }
  cudaGetDevice(&h->dev);
  const size_t n = (size_t)total;
  const int nblk = (int)((A.nbucket + kScanPerBlock - 1) / kScanPerBlock);
  cudaError_t e = cudaSuccess;
  auto al = [&](cudaError_t r) {
    if (e == cudaSuccess) e = r;
  };
  al(dalloc(h, &A.x, 3 * n));
  al(dalloc(h, &A.ph, 3 * n));
  al(dalloc(h, &A.pk, 3 * n));
  al(dalloc(h, &A.xref, 3 * n));
  {
    void* f = nullptr;
    al(h->precision == MD_PREC_FP64 ? dalloc(h, reinterpret_cast<double4_32a**>(&f), n)
                                    : dalloc(h, reinterpret_cast<float4**>(&f), n));
    A.f = f;
    void* r = nullptr;
    al(h->precision == MD_PREC_FP64 ? dalloc(h, reinterpret_cast<double4_32a**>(&r), n)
                                    : dalloc(h, reinterpret_cast<float4**>(&r), n));
    A.rec = r;
    if (h->precision != MD_PREC_FP64) al(dalloc(h, &A.rec_lo, n));
  }
  al(dalloc(h, &A.meta, n));
  if (h->excl) al(dalloc(h, &A.mol, n));
  al(dalloc(h, &A.cell, n));
  al(dalloc(h, &A.rank, n));
  al(dalloc(h, &A.count, A.nbucket));
  al(dalloc(h, &A.start, (size_t)A.nbucket + 1));
  al(dalloc(h, &A.blocksum, (size_t)nblk));
  al(dalloc(h, &A.tile_state, (size_t)nblk));
  al(dalloc(h, &A.scan, 1));
  al(dalloc(h, &A.gbar, 1));
  al(dalloc(h, &A.rb_sum, (size_t)kRebuildMaxBlocks));
  // order keys: (system, Morton code of the cell) packed into at most 2^20 keys
  {
    int maxnc = 1;
    for (int sy = 0; sy < nsys; ++sy)
      for (int d = 0; d < 3; ++d) maxnc = std::max(maxnc, h->sys[sy].nc[d]);
    uint32_t cbits = 0;
    while ((1 << cbits) < maxnc) ++cbits;
    const uint32_t coord_shift = cbits > 10 ? cbits - 10 : 0;
    const uint32_t mbits = 3 * std::min<uint32_t>(cbits, 10);
    uint32_t sbits = 0;
    while ((1u << sbits) < (uint32_t)nsys) ++sbits;
    const uint32_t kKeyBits = 20;
    uint32_t keep = sbits >= kKeyBits ? 0 : std::min(mbits, kKeyBits - sbits);
    h->order_coord_shift = coord_shift;
    h->order_morton_drop = mbits - keep;
    h->order_sys_shift = keep;
    const uint64_t nkeys = (uint64_t)nsys << keep;
    h->O = A;
    h->O.nbucket = (uint32_t)std::min<uint64_t>(nkeys, uint64_t(1) << 31);
    const size_t ot = (h->O.nbucket + kScanPerBlock - 1) / kScanPerBlock;
    al(dalloc(h, &h->O.count, h->O.nbucket));
    al(dalloc(h, &h->O.start, (size_t)h->O.nbucket + 1));
    al(dalloc(h, &h->O.tile_state, ot));
    al(dalloc(h, &h->O.scan, 1));
  }
  al(dalloc(h, &A.stag, n));
  al(dalloc(h, &A.stag_tmp, n));
  al(dalloc(h, &A.slot_of, n));
  al(dalloc(h, &h->d_order, n));
  al(dalloc(h, &h->d_res_order, (size_t)nsys));
  al(dalloc(h, &h->d_res_next, 1));
  al(dalloc(h, &A.scell, n));
  SysDev* d_sys = nullptr;
  al(dalloc(h, &d_sys, (size_t)nsys));
  A.sys = d_sys;
  TypeTable* d_types = nullptr;
  al(dalloc(h, &d_types, 1));
  A.types = d_types;
  al(dalloc(h, &A.status, 1));
  al(dalloc(h, &A.step, 1));
  al(dalloc(h, &A.mode, 1));
  al(dalloc(h, &h->d_first, (size_t)nsys));
  al(dalloc(h, &A.sys_free, (size_t)nsys));
  al(dalloc(h, &h->d_stage, 9 * n));
  al(dalloc(h, &h->d_stage_i, 2 * n));
  al(dalloc(h, &h->d_stage_u8, n));
  al(dalloc(h, &h->d_resid, 3));
  al(dalloc(h, &h->d_obs, 8 * (size_t)nsys));
  if (e == cudaSuccess) e = cudaMallocHost(&h->h_status, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMallocHost(&h->h_resid, 3 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMemcpy(d_sys, h->sys.data(), sizeof(SysDev) * nsys, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_types, &h->types, sizeof(TypeTable), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(h->d_first, h->first.data(), sizeof(int64_t) * nsys, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(A.count, 0, sizeof(uint32_t) * std::max<size_t>(A.nbucket, 1));
  if (e == cudaSuccess) e = cudaMemset(A.tile_state, 0, sizeof(unsigned long long) * (size_t)nblk);
  if (e == cudaSuccess) e = cudaMemset(A.scan, 0, sizeof(ScanCtl));
  if (e == cudaSuccess) e = cudaMemset(A.gbar, 0, sizeof(GridBar));
  if (e == cudaSuccess) e = cudaMemset(h->O.count, 0, sizeof(uint32_t) * h->O.nbucket);
  if (e == cudaSuccess)
    e = cudaMemset(h->O.tile_state, 0,
                   sizeof(unsigned long long) * ((h->O.nbucket + kScanPerBlock - 1) / kScanPerBlock));
  if (e == cudaSuccess) e = cudaMemset(h->O.scan, 0, sizeof(ScanCtl));
  if (e == cudaSuccess) {
    const uint32_t nn = (uint32_t)total;
    e = cudaMemcpy(h->O.start + h->O.nbucket, &nn, sizeof(uint32_t), cudaMemcpyHostToDevice);
  }
  h->O.status = A.status;  // the order scan reports through the handle's status word
  h->O.n = A.n;
  if (h->has_pairs && total > 0) A.order = h->d_order;
  if (e == cudaSuccess) e = cudaMemset(A.status, 0, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemset(A.step, 0, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(A.mode, 0, sizeof(int32_t));
  if (e == cudaSuccess) {
    const uint32_t nn = (uint32_t)total;
    e = cudaMemcpy(A.start + A.nbucket, &nn, sizeof(uint32_t), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    std::string m = std::string("allocation / upload failed: ") + cudaGetErrorString(e);
    md_destroy(h);
    return fail(nullptr, MD_ERR_CUDA, m);
  }
  if (e == cudaSuccess) {  // resident work list: largest systems first
    std::vector<int32_t> ord((size_t)nsys);
    for (int q = 0; q < nsys; ++q) ord[(size_t)q] = q;
    std::stable_sort(ord.begin(), ord.end(), [&](int32_t a, int32_t b) { return n_per_sys[a] > n_per_sys[b]; });
    e = cudaMemcpy(h->d_res_order, ord.data(), sizeof(int32_t) * (size_t)nsys, cudaMemcpyHostToDevice);
    for (int32_t q : ord) {
      h->res_n_sorted.push_back(n_per_sys[q]);
      h->res_t_sorted.push_back(h->sys[(size_t)q].res_t);
    }
  }
  if (e != cudaSuccess) {
    std::string m = std::string("allocation / upload failed: ") + cudaGetErrorString(e);
    md_destroy(h);
    return fail(nullptr, MD_ERR_CUDA, m);
  }
  *out = h;
  return MD_OK;
}

int md_set_stream(md_handle* h, void* cuda_stream) {
  if (!h) return MD_ERR_INVALID_ARG;
  h->user_stream = static_cast<cudaStream_t>(cuda_stream);
  return MD_OK;
}

static int set_state_common(md_handle* h, const double* d_x, const double* d_v, const int32_t* d_type,
                            const int32_t* d_mol, const uint8_t* d_con, uint64_t step0) {
  cudaStream_t st = h->stream();
  CK(h, cudaMemsetAsync(h->A.sys_free, 0, sizeof(int32_t) * (size_t)h->nsys, st));
  CK(h, launch_build_meta(h->A, h->d_first, h->nsys, d_type, d_con, d_mol, 0, st));
  CK(h, launch_set_state(h->A, d_x, d_v, st));
  const unsigned long long k = step0;
  CK(h, cudaMemcpyAsync(h->A.step, &k, sizeof(k), cudaMemcpyHostToDevice, st));
  CK(h, cudaMemsetAsync(h->A.mode, 0, sizeof(int32_t), st));
  if (h->A.noise_k) CK(h, cudaMemsetAsync(h->A.noise_k, 0xff, sizeof(unsigned long long), st));  // none stored
  int rc = rebuild_cells(h);
  if (rc) return rc;
  h->state_set = true;
  rc = check_device_status(h);
  if (rc != MD_OK) h->state_set = false;
  return rc;
}

int md_set_state(md_handle* h, const double* x, const double* v, const int32_t* type, const int32_t* mol,
                 const uint8_t* constrained, uint64_t step0) {
  if (!h) return MD_ERR_INVALID_ARG;
  if (h->n > 0 && !x) return fail(h, MD_ERR_INVALID_ARG, "x must not be NULL");
  CK(h, cudaSetDevice(h->dev));
  const size_t n = (size_t)h->n;
  cudaStream_t st = h->stream();
  if (n > 0) {
    CK(h, cudaMemcpyAsync(h->d_stage, x, 3 * n * sizeof(double), cudaMemcpyHostToDevice, st));
    if (v) CK(h, cudaMemcpyAsync(h->d_stage + 3 * n, v, 3 * n * sizeof(double), cudaMemcpyHostToDevice, st));
    if (type) CK(h, cudaMemcpyAsync(h->d_stage_i, type, n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    if (mol) CK(h, cudaMemcpyAsync(h->d_stage_i + n, mol, n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    if (constrained) CK(h, cudaMemcpyAsync(h->d_stage_u8, constrained, n, cudaMemcpyHostToDevice, st));
  }
  return set_state_common(h, h->d_stage, v ? h->d_stage + 3 * n : nullptr, type ? h->d_stage_i : nullptr,
                          mol ? h->d_stage_i + n : nullptr, constrained ? h->d_stage_u8 : nullptr, step0);
}

int md_set_state_device(md_handle* h, const double* d_x, const double* d_v, const int32_t* d_type,
                        const int32_t* d_mol, const uint8_t* d_con, uint64_t step0) {
  if (!h) return MD_ERR_INVALID_ARG;
  if (h->n > 0 && !d_x) return fail(h, MD_ERR_INVALID_ARG, "d_x must not be NULL");
  CK(h, cudaSetDevice(h->dev));
  return set_state_common(h, d_x, d_v, d_type, d_mol, d_con, step0);
}

int md_restore(md_handle* h, const double* x, const double* p_half, uint64_t step) {
  int rc = require_state(h);
  if (rc) return rc;
  if (h->n > 0 && (!x || !p_half)) return fail(h, MD_ERR_INVALID_ARG, "x and p_half must not be NULL");
  const size_t n = (size_t)h->n;
  cudaStream_t st = h->stream();
  if (n > 0) {
    CK(h, cudaMemcpyAsync(h->d_stage, x, 3 * n * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(h, cudaMemcpyAsync(h->d_stage + 3 * n, p_half, 3 * n * sizeof(double), cudaMemcpyHostToDevice, st));
  }
  CK(h, launch_restore(h->A, h->d_stage, h->d_stage + 3 * n, st));
  const unsigned long long k = step;
  const int32_t one = 1;
  CK(h, cudaMemcpyAsync(h->A.step, &k, sizeof(k), cudaMemcpyHostToDevice, st));
  CK(h, cudaMemcpyAsync(h->A.mode, &one, sizeof(one), cudaMemcpyHostToDevice, st));
  if (h->A.noise_k) CK(h, cudaMemsetAsync(h->A.noise_k, 0xff, sizeof(unsigned long long), st));  // none stored
  rc = rebuild_cells(h);
  if (rc) return rc;
  return check_device_status(h);
}

int md_step(md_handle* h, int64_t nsteps) {
  int rc = require_state(h);
  if (rc) return rc;
  if (nsteps < 0) return fail(h, MD_ERR_INVALID_ARG, "nsteps must be >= 0");
  h->last_launches = 0;
  if (nsteps == 0) return MD_OK;
  if (h->cells_stale) {  // the previous step's cell list did not complete
    rc = rebuild_cells(h);
    if (rc) return rc;
    h->cells_stale = false;
  }
  if (h->engine == 1) return resident_steps(h, nsteps);
  rc = build_graph(h);
  if (rc) return rc;
  int64_t extra = 0;
  for (int64_t s = 0; s < nsteps; ++s) {
    CK(h, cudaGraphLaunch(h->graph, h->stream()));
    if (h->has_pairs && h->A.order && !h->A.nl_dirty && ++h->steps_since_order >= kOrderEvery) {
      // any permutation is a valid visiting order; a fresh one keeps it spatial
      CK(h, launch_order(h->A, h->O, h->order_coord_shift, h->order_morton_drop, h->order_sys_shift, h->d_order,
                     h->stream()));
      h->steps_since_order = 0;
      extra += 3;
    }
  }
  const StepKernel* ks;
  h->last_launches = nsteps * step_kernels(h, &ks) + extra;
  return MD_OK;
}

int md_profile_step(md_handle* h, int64_t nsteps, double* kernel_ms, int32_t max_kernels,
                    int32_t* n_kernels) {
  int rc = require_state(h);
  if (rc) return rc;
  if (nsteps < 1 || !kernel_ms || max_kernels < 1) return fail(h, MD_ERR_INVALID_ARG, "bad profile arguments");
  if (h->engine == 1) {  // resident engine: its launches per step, then the global cell-list rebuild per call
    cudaEvent_t ev[3];
    for (auto& e : ev) CK(h, cudaEventCreate(&e));
    cudaStream_t st = h->stream();
    int status = MD_OK;
    int64_t launches = 0;
    cudaError_t e = cudaEventRecord(ev[0], st);
    if (e == cudaSuccess) e = enqueue_resident(h, nsteps, st, &launches);
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], st);
    if (e != cudaSuccess) status = cuda_fail(h, e, "resident");
    if (status == MD_OK) status = rebuild_cells(h);
    if (status == MD_OK) {
      e = cudaEventRecord(ev[2], st);
      if (e == cudaSuccess) e = cudaEventSynchronize(ev[2]);
      if (e != cudaSuccess) status = cuda_fail(h, e, "profile event");
    }
    float ms[2] = {0.f, 0.f};
    if (status == MD_OK) {
      cudaEventElapsedTime(&ms[0], ev[0], ev[1]);
      cudaEventElapsedTime(&ms[1], ev[1], ev[2]);
    }
    for (auto& ee : ev) cudaEventDestroy(ee);
    if (status != MD_OK) return status;
    kernel_ms[0] = ms[0] / (double)nsteps;
    if (max_kernels > 1) kernel_ms[1] = ms[1] / (double)nsteps;
    if (n_kernels) *n_kernels = 2;
    h->last_launches = launches + kRebuildLaunches;
    return check_device_status(h);
  }
  const StepKernel* ks;
  const int nk = step_kernels(h, &ks);
  std::vector<cudaEvent_t> ev((size_t)nk + 1);
  for (auto& e : ev) CK(h, cudaEventCreate(&e));
  std::vector<double> acc((size_t)nk, 0.0);
  cudaStream_t st = h->stream();
  int status = MD_OK;
  for (int64_t s = 0; s < nsteps && status == MD_OK; ++s) {
    for (int i = 0; i < nk; ++i) {
      cudaError_t e = cudaEventRecord(ev[i], st);
      if (e == cudaSuccess) e = ks[i].fn(h, st);
      if (e != cudaSuccess) {
        status = cuda_fail(h, e, ks[i].name);
        break;
      }
    }
    if (status != MD_OK) break;
    cudaError_t e = cudaEventRecord(ev[nk], st);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[nk]);
    if (e != cudaSuccess) {
      status = cuda_fail(h, e, "profile event");
      break;
    }
    for (int i = 0; i < nk; ++i) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[i], ev[i + 1]);
      acc[i] += ms;
    }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  if (status != MD_OK) return status;
  const int m = std::min<int>(nk, max_kernels);
  for (int i = 0; i < m; ++i) kernel_ms[i] = acc[i] / (double)nsteps;
  if (n_kernels) *n_kernels = nk;
  h->last_launches = nsteps * nk;
  return check_device_status(h);
}

const char* md_profile_kernel_name(md_handle* h, int32_t i) {
  if (!h) return "";
  if (h->engine == 1) return i == 0 ? "resident" : (i == 1 ? "rebuild" : "");
  const StepKernel* ks;
  const int nk = step_kernels(h, &ks);
  return (i >= 0 && i < nk) ? ks[i].name : "";
}

int md_set_neighbor_list(md_handle* h, double skin, int32_t max_neighbors) {
  if (!h) return MD_ERR_INVALID_ARG;
  if (!(skin > 0.0)) {  // off: back to the per-step cell list
    if (h->A.nl_dirty) {
      h->A.nl_dirty = nullptr;
      if (h->state_set) {
        int rc = rebuild_cells(h);
        if (rc) return rc;
      }
    }
  } else {
    if (!h->has_pairs) return fail(h, MD_ERR_INVALID_ARG, "the neighbour list needs pair interactions");
    if (!std::isfinite(skin) || max_neighbors < 1 || max_neighbors > 4096)
      return fail(h, MD_ERR_INVALID_ARG, "skin must be finite and max_neighbors in 1..4096");
    if (h->n >= (int64_t(1) << 27)) return fail(h, MD_ERR_INVALID_ARG, "the neighbour list holds at most 2^27 particles");
    double rcmax = 0.0;
    for (int a = 0; a < MD_MAX_TYPES; ++a)
      for (int b = 0; b < MD_MAX_TYPES; ++b) rcmax = std::max(rcmax, std::sqrt(h->types.rc2[a][b]));
    for (const SysDev& S : h->sys)
      for (int d = 0; d < 3; ++d)
        if ((S.nc[d] > 1 || S.periodic[d]) && S.cs[d] < rcmax + skin)
          return fail(h, MD_ERR_INVALID_ARG,
                      "cell edge " + std::to_string(S.cs[d]) + " is below r_c + skin = " +
                          std::to_string(rcmax + skin) + ": create the handle with cell_size >= r_c + skin");
    DevArrays& A = h->A;
    if (max_neighbors > h->nl_capacity) {  // the arrays of a smaller list stay allocated until md_destroy
      const size_t n = (size_t)h->n;
      cudaError_t e = cudaSuccess;
      if (!h->d_nl_dirty) e = dalloc(h, &h->d_nl_dirty, 1);
      if (e == cudaSuccess) e = dalloc(h, &A.nl, (size_t)max_neighbors * n);
      if (e == cudaSuccess) e = dalloc(h, &A.nl_cnt, n);
      if (e == cudaSuccess) e = dalloc(h, &A.nl_pk, (size_t)max_neighbors * n);
      if (e == cudaSuccess) e = dalloc(h, &A.nl_off, n);
      if (e == cudaSuccess) e = dalloc(h, &A.smeta, n);
      if (e == cudaSuccess) e = dalloc(h, &A.xb, 3 * n);
      if (e == cudaSuccess && !A.nl_builds) {
        e = dalloc(h, &A.nl_builds, 1);
        if (e == cudaSuccess) e = cudaMemsetAsync(A.nl_builds, 0, sizeof(unsigned long long), h->stream());
      }
      if (e == cudaSuccess)
        e = h->precision == MD_PREC_FP64 ? dalloc(h, reinterpret_cast<double4_32a**>(&A.rec0), n)
                                         : dalloc(h, reinterpret_cast<float4**>(&A.rec0), n);
      if (e == cudaSuccess && h->precision != MD_PREC_FP64) e = dalloc(h, &A.rec0_lo, n);
      if (e == cudaSuccess && h->precision != MD_PREC_FP64) e = dalloc(h, &A.noise, n);
      if (e == cudaSuccess && h->precision != MD_PREC_FP64 && !A.noise_k) {
        e = dalloc(h, &A.noise_k, 1);
        if (e == cudaSuccess) e = cudaMemsetAsync(A.noise_k, 0xff, sizeof(unsigned long long), h->stream());
      }
      if (e != cudaSuccess) return cuda_fail(h, e, "neighbour list allocation");
      h->nl_capacity = max_neighbors;
    }
    A.nl_max = max_neighbors;
    A.nl_skin = skin;
    A.nl_half_skin2 = (float)(0.25 * skin * skin);
    A.nl_dirty = h->d_nl_dirty;
    if (h->state_set) {
      int rc = rebuild_cells(h);
      if (rc) return rc;
    }
  }
  if (h->graph) {  // the captured step used the old mode
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  return check_device_status(h);
}

int md_set_option(md_handle* h, int32_t key, int64_t value) {
  if (!h) return MD_ERR_INVALID_ARG;
  switch (key) {
    case MD_OPT_PAIR_LANES:
      if (value != 1 && value != 2 && value != 4 && value != 8)
        return fail(h, MD_ERR_INVALID_ARG, "pair lanes must be 1, 2, 4 or 8");
      h->A.pair_lanes = (int32_t)value;
      break;
    case MD_OPT_PAIR_ORDER:
      if (value != 0 && value != 1) return fail(h, MD_ERR_INVALID_ARG, "pair order must be 0 or 1");
      h->A.order = (value && h->has_pairs && h->n > 0) ? h->d_order : nullptr;
      if (h->A.order && h->state_set) {
        CK(h, launch_order(h->A, h->O, h->order_coord_shift, h->order_morton_drop, h->order_sys_shift,
                           h->d_order, h->stream()));
        h->steps_since_order = 0;
      }
      break;
    case MD_OPT_ENGINE: {
      if (value != 0 && value != 1) return fail(h, MD_ERR_INVALID_ARG, "engine must be 0 or 1");
      if (value == 1) {
        const std::string why = plan_resident(h, h->res_threads);
        if (!why.empty()) return fail(h, MD_ERR_INVALID_ARG, why);
      }
      h->engine = (int)value;
      break;
    }
    case MD_OPT_RESIDENT_THREADS: {
      if (value != 0 && (value < 64 || value > kResidentMaxThreads || value % 32 != 0))
        return fail(h, MD_ERR_INVALID_ARG, "resident threads must be 0 (automatic) or a multiple of 32 in 64..512");
      if (h->engine == 1) {
        const std::string why = plan_resident(h, (int)value);
        if (!why.empty()) {
          plan_resident(h, h->res_threads);  // keep the previous plan
          return fail(h, MD_ERR_INVALID_ARG, why);
        }
      }
      h->res_threads = (int)value;
      break;
    }
    case MD_OPT_RESIDENT_STEPS:
      if (value < 1 || value > 100000) return fail(h, MD_ERR_INVALID_ARG, "steps per launch must be in 1..100000");
      h->res_steps_per_launch = value;
      break;
    case MD_OPT_PAIR_QUEUE:
      if (value != 0 && value != 1) return fail(h, MD_ERR_INVALID_ARG, "pair queue must be 0 or 1");
      h->A.pair_queue = (int32_t)value;
      break;
    case MD_OPT_LIST_WARP:
      if (value != 8 && value != 16 && value != 32)
        return fail(h, MD_ERR_INVALID_ARG, "particles per warp of the list walk must be 8, 16 or 32");
      h->A.list_warp = (int32_t)value;
      break;
    case MD_OPT_STORE_NOISE:
      if (value != 0 && value != 1) return fail(h, MD_ERR_INVALID_ARG, "store noise must be 0 or 1");
      h->A.store_noise = (int32_t)value;
      if (h->A.noise_k) CK(h, cudaMemsetAsync(h->A.noise_k, 0xff, sizeof(unsigned long long), h->stream()));
      break;
    case MD_OPT_FUSED_REBUILD:
      if (value != 0 && value != 1) return fail(h, MD_ERR_INVALID_ARG, "fused rebuild must be 0 or 1");
      h->fused_rebuild = (int)value;
      h->rebuild_ctas = 0;
      break;
    case MD_OPT_SPIN_LIMIT:
      if (value < 0 || value > 0x7fffffff) return fail(h, MD_ERR_INVALID_ARG, "spin limit must be in 0..2^31-1");
      h->A.spin_limit = (uint32_t)value;
      break;
    case MD_OPT_PAIR_TILE:
      if (value != 0 && value != 8 && value != 16 && value != 32)
        return fail(h, MD_ERR_INVALID_ARG, "pair tile must be 0, 8, 16 or 32");
      if (value != 0 && h->has_pairs && h->A.hashed)
        return fail(h, MD_ERR_INVALID_ARG, "the cell-tiled pair kernel needs a grid of at most max(2^20, 4N) cells");
      h->A.pair_tile = (int32_t)value;
      break;
    default:
      return fail(h, MD_ERR_INVALID_ARG, "unknown option");
  }
  if (h->graph) {  // the captured step used the old setting
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  return MD_OK;
}

int md_get_option(md_handle* h, int32_t key, int64_t* value) {
  if (!h || !value) return MD_ERR_INVALID_ARG;
  switch (key) {
    case MD_OPT_PAIR_LANES: *value = h->A.pair_lanes; return MD_OK;
    case MD_OPT_PAIR_ORDER: *value = h->A.order ? 1 : 0; return MD_OK;
    case MD_OPT_ENGINE: *value = h->engine; return MD_OK;
    case MD_OPT_RESIDENT_THREADS: *value = h->res_threads; return MD_OK;
    case MD_OPT_RESIDENT_STEPS: *value = h->res_steps_per_launch; return MD_OK;
    case MD_OPT_PAIR_TILE: *value = h->A.pair_tile; return MD_OK;
    case MD_OPT_SPIN_LIMIT: *value = h->A.spin_limit; return MD_OK;
    case MD_OPT_PAIR_QUEUE: *value = h->A.pair_queue; return MD_OK;
    case MD_OPT_FUSED_REBUILD: *value = h->fused_rebuild; return MD_OK;
    case MD_OPT_LIST_WARP: *value = h->A.list_warp; return MD_OK;
    case MD_OPT_STORE_NOISE: *value = h->A.store_noise; return MD_OK;
    case MD_OPT_NLIST_BUILDS: {
      unsigned long long b = 0;
      if (h->A.nl_builds) {
        CK(h, cudaMemcpyAsync(&b, h->A.nl_builds, sizeof(b), cudaMemcpyDeviceToHost, h->stream()));
        CK(h, cudaStreamSynchronize(h->stream()));
      }
      *value = (int64_t)b;
      return MD_OK;
    }
    default: return fail(h, MD_ERR_INVALID_ARG, "unknown option");
  }
}

int md_sync(md_handle* h) {
  if (!h) return MD_ERR_INVALID_ARG;
  CK(h, cudaSetDevice(h->dev));
  return check_device_status(h);
}

int md_status(md_handle* h, uint32_t* flags) {
  if (!h || !flags) return MD_ERR_INVALID_ARG;
  CK(h, cudaSetDevice(h->dev));
  CK(h, cudaMemcpyAsync(h->h_status, h->A.status, sizeof(uint32_t), cudaMemcpyDeviceToHost, h->stream()));
  CK(h, cudaStreamSynchronize(h->stream()));
  *flags = *h->h_status & 0xffu;
  CK(h, cudaMemsetAsync(h->A.status, 0, sizeof(uint32_t), h->stream()));
  CK(h, cudaStreamSynchronize(h->stream()));
  return MD_OK;
}

int md_get_state_device(md_handle* h, double* d_x, double* d_v, double* d_p_half) {
  int rc = require_state(h);
  if (rc) return rc;
  if (d_v) {
    rc = momenta_now(h);
    if (rc) return rc;
  }
  CK(h, launch_get_state(h->A, d_x, d_v, d_p_half, h->stream()));
  return check_device_status(h);
}

int md_get_state(md_handle* h, double* x, double* v, double* p_half, uint64_t* step) {
  int rc = require_state(h);
  if (rc) return rc;
  const size_t n = (size_t)h->n;
  cudaStream_t st = h->stream();
  double* sx = h->d_stage;
  double* sv = h->d_stage + 3 * n;
  double* sp = h->d_stage + 6 * n;
  if (v) {
    rc = momenta_now(h);
    if (rc) return rc;
  }
  CK(h, launch_get_state(h->A, x ? sx : nullptr, v ? sv : nullptr, p_half ? sp : nullptr, st));
  if (x && n) CK(h, cudaMemcpyAsync(x, sx, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (v && n) CK(h, cudaMemcpyAsync(v, sv, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (p_half && n) CK(h, cudaMemcpyAsync(p_half, sp, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, st));
  unsigned long long k = 0;
  CK(h, cudaMemcpyAsync(&k, h->A.step, sizeof(k), cudaMemcpyDeviceToHost, st));
  CK(h, cudaStreamSynchronize(st));
  if (step) *step = k;
  return check_device_status(h);
}

int md_forces(md_handle* h, double* f_out, double* u_out) {
  int rc = require_state(h);
  if (rc) return rc;
  const size_t n = (size_t)h->n;
  cudaStream_t st = h->stream();
  rc = forces_now(h);
  if (rc) return rc;
  CK(h, launch_get_forces(h->A, h->precision, h->d_stage, h->d_stage + 3 * n, st));
  if (f_out && n) CK(h, cudaMemcpyAsync(f_out, h->d_stage, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (u_out && n) CK(h, cudaMemcpyAsync(u_out, h->d_stage + 3 * n, n * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(h, cudaStreamSynchronize(st));
  return check_device_status(h);
}

int md_constraint_residual(md_handle* h, double* max_g_over_gradg, double* max_abs_g, double* max_n_dot_v) {
  int rc = require_state(h);
  if (rc) return rc;
  rc = momenta_now(h);
  if (rc) return rc;
  cudaStream_t st = h->stream();
  CK(h, launch_residual(h->A, h->d_resid, st));
  CK(h, cudaMemcpyAsync(h->h_resid, h->d_resid, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
  CK(h, cudaStreamSynchronize(st));
  double r[3];
  std::memcpy(r, h->h_resid, sizeof(r));
  if (max_g_over_gradg) *max_g_over_gradg = r[0];
  if (max_abs_g) *max_abs_g = r[1];
  if (max_n_dot_v) *max_n_dot_v = r[2];
  return check_device_status(h);
}

int md_observables(md_handle* h, md_obs* out, int32_t max_systems, int32_t* n_written) {
  int rc = require_state(h);
  if (rc) return rc;
  if (!out || max_systems < 0) return fail(h, MD_ERR_INVALID_ARG, "out must not be NULL");
  rc = momenta_now(h);
  if (rc) return rc;
  cudaStream_t st = h->stream();
  CK(h, launch_observables(h->A, h->precision, h->d_obs, st));
  std::vector<double> o(8 * (size_t)h->nsys);
  unsigned long long k = 0;
  CK(h, cudaMemcpyAsync(o.data(), h->d_obs, o.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(h, cudaMemcpyAsync(&k, h->A.step, sizeof(k), cudaMemcpyDeviceToHost, st));
  CK(h, cudaStreamSynchronize(st));
  const int m = std::min<int>(max_systems, h->nsys);
  for (int s = 0; s < m; ++s) {
    const double* q = &o[8 * (size_t)s];
    md_obs& r = out[s];
    r.step = k;
    r.n = (int64_t)q[7];
    r.ndof = (int64_t)q[4];
    r.kinetic = q[0];
    r.potential = q[1];
    r.kT = q[4] > 0 ? 2.0 * q[0] / q[4] : 0.0;
    r.max_g_over_gradg = q[5];
    r.max_n_dot_v = q[6];
    r.msd = q[7] > 0 ? q[2] / q[7] : 0.0;
    r.r0_dot_rt = (h->sys[s].kind == MD_SURF_SPHERE && q[7] > 0) ? q[3] / q[7] : 0.0;
  }
  if (n_written) *n_written = m;
  return check_device_status(h);
}

int md_info(md_handle* h, int64_t* n, int32_t* nsys, uint64_t* step) {
  if (!h) return MD_ERR_INVALID_ARG;
  if (n) *n = h->n;
  if (nsys) *nsys = h->nsys;
  if (step) {
    CK(h, cudaSetDevice(h->dev));
    unsigned long long k = 0;
    CK(h, cudaMemcpyAsync(&k, h->A.step, sizeof(k), cudaMemcpyDeviceToHost, h->stream()));
    CK(h, cudaStreamSynchronize(h->stream()));
    *step = k;
  }
  return MD_OK;
}

int md_last_launch_count(md_handle* h, int64_t* launches) {
  if (!h || !launches) return MD_ERR_INVALID_ARG;
  *launches = h->last_launches;
  return MD_OK;
}

int md_grid_info(md_handle* h, int32_t sys, double lo[3], double cs[3], int32_t nc[3], uint32_t* base,
                 int32_t* hashed) {
  if (!h || sys < 0 || sys >= h->nsys) return MD_ERR_INVALID_ARG;
  const SysDev& S = h->sys[sys];
  for (int d = 0; d < 3; ++d) {
    if (lo) lo[d] = S.grid_lo[d];
    if (cs) cs[d] = S.cs[d];
    if (nc) nc[d] = S.nc[d];
  }
  if (base) *base = S.cell_base;
  if (hashed) *hashed = h->A.hashed ? h->A.log_t : 0;
  return MD_OK;
}

int md_cell_list(md_handle* h, uint32_t* sorted_ids, uint32_t* sorted_cells, uint32_t* bucket_start,
                 uint32_t* nbucket) {
  int rc = require_state(h);
  if (rc) return rc;
  if (nbucket) *nbucket = h->has_pairs ? h->A.nbucket : 0;
  if (!h->has_pairs) return MD_OK;
  cudaStream_t st = h->stream();
  const size_t n = (size_t)h->n;
  if (sorted_ids && n) CK(h, cudaMemcpyAsync(sorted_ids, h->A.stag, n * 4, cudaMemcpyDeviceToHost, st));
  if (sorted_cells && n) CK(h, cudaMemcpyAsync(sorted_cells, h->A.scell, n * 4, cudaMemcpyDeviceToHost, st));
  if (bucket_start)
    CK(h, cudaMemcpyAsync(bucket_start, h->A.start, ((size_t)h->A.nbucket + 1) * 4, cudaMemcpyDeviceToHost, st));
  CK(h, cudaStreamSynchronize(st));
  return check_device_status(h);
}

int md_check_conversions(const double* in, int64_t n, float* out_f32, double* out_f64) {
  if (n < 0 || (n > 0 && (!in || !out_f32 || !out_f64))) return fail(nullptr, MD_ERR_INVALID_ARG, "bad arguments");
  if (n == 0) return MD_OK;
  double* d_in = nullptr;
  double* d_d = nullptr;
  float* d_f = nullptr;
  const size_t nb = (size_t)n;
  cudaError_t e = cudaMalloc(&d_in, nb * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&d_d, nb * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&d_f, nb * sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpy(d_in, in, nb * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = launch_check_conversions(d_in, n, d_f, d_d, 0);
  if (e == cudaSuccess) e = cudaMemcpy(out_f32, d_f, nb * sizeof(float), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(out_f64, d_d, nb * sizeof(double), cudaMemcpyDeviceToHost);
  cudaFree(d_in);
  cudaFree(d_d);
  cudaFree(d_f);
  if (e != cudaSuccess) return fail(nullptr, MD_ERR_CUDA, std::string("conversion check: ") + cudaGetErrorString(e));
  return MD_OK;
}

int md_measure_fma_peak(int32_t precision, int32_t trials, double* fma_per_s) {
  if ((precision != MD_PREC_FP64 && precision != MD_PREC_MIXED) || trials < 1 || !fma_per_s)
    return fail(nullptr, MD_ERR_INVALID_ARG, "precision must be MD_PREC_FP64 or MD_PREC_MIXED, trials >= 1");
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // long enough to time (~ms), short enough to stay a probe
  const int blocks = 16 * std::max(sms, 1), iters = precision == MD_PREC_FP64 ? 256 : 16384;
  cudaStream_t st = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (e == cudaSuccess) e = launch_fma_probe(precision == MD_PREC_FP64 ? 0 : 1, blocks, iters, st);  // warm-up
  double best = 0.0;
  for (int t = 0; t < trials && e == cudaSuccess; ++t) {
    e = cudaEventRecord(a, st);
    if (e == cudaSuccess) e = launch_fma_probe(precision == MD_PREC_FP64 ? 0 : 1, blocks, iters, st);
    if (e == cudaSuccess) e = cudaEventRecord(b, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e == cudaSuccess && ms > 0.f) best = std::max(best, (double)blocks * 256.0 * 8.0 * iters / (ms * 1e-3));
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (st) cudaStreamDestroy(st);
  if (e != cudaSuccess) return fail(nullptr, MD_ERR_CUDA, std::string("peak probe: ") + cudaGetErrorString(e));
  *fma_per_s = best;
  return MD_OK;
}

const char* md_last_error(md_handle* h) {
  if (!h) return g_create_err.c_str();
  return h->err.c_str();
}

void md_destroy(md_handle* h) {
  if (!h) return;
  cudaSetDevice(h->dev);
  if (h->own_stream) cudaStreamSynchronize(h->own_stream);
  if (h->user_stream) cudaStreamSynchronize(h->user_stream);
  if (h->graph) cudaGraphExecDestroy(h->graph);
  for (void* p : h->allocs) cudaFree(p);
  if (h->h_status) cudaFreeHost(h->h_status);
  if (h->h_resid) cudaFreeHost(h->h_resid);
  if (h->own_stream) cudaStreamDestroy(h->own_stream);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  delete h;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// md_forces_noalloc: forces of one system without any device allocation.
//
// For callers that cannot allocate device memory at the point where they need
// forces -- a host thread working while a CUDA graph is being captured in
// global mode (cudaMalloc is not permitted then), or an application whose
// device memory is entirely reserved by its own allocator. All scratch (cell
// list, records, tables) lives in one fixed-size array in device global
// memory, reserved when the library's device code is loaded; every device that
// loads the library keeps it until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr int64_t kNaMaxParticles = 65536;
constexpr uint32_t kNaMaxBuckets = 1u << 18;

constexpr size_t na_align(size_t v) { return (v + 255) & ~size_t(255); }

// Byte offsets of the regions of the scratch array (each 256-byte aligned).
struct NaLayout {
  static constexpr size_t N = (size_t)kNaMaxParticles, T = (size_t)kNaMaxBuckets;
  static constexpr size_t x = 0;
  static constexpr size_t f = x + na_align(3 * N * sizeof(double));
  static constexpr size_t rec = f + na_align(N * sizeof(double4_32a));
  static constexpr size_t rec_lo = rec + na_align(N * sizeof(double4_32a));
  static constexpr size_t meta = rec_lo + na_align(N * sizeof(float4));
  static constexpr size_t mol = meta + na_align(N * 4);
  static constexpr size_t cell = mol + na_align(N * 4);
  static constexpr size_t rank = cell + na_align(N * 4);
  static constexpr size_t stag = rank + na_align(N * 4);
  static constexpr size_t stag_tmp = stag + na_align(N * 4);
  static constexpr size_t scell = stag_tmp + na_align(N * 4);
  static constexpr size_t count = scell + na_align(N * 4);
  static constexpr size_t start = count + na_align(T * 4);
  static constexpr size_t blocksum = start + na_align((T + 1) * 4);
  static constexpr size_t tile_state = blocksum + na_align((T / kScanPerBlock + 1) * 4);
  static constexpr size_t scan = tile_state + na_align((T / kScanPerBlock + 1) * 8);
  static constexpr size_t sys = scan + 256;
  static constexpr size_t types = sys + na_align(sizeof(SysDev));
  static constexpr size_t status = types + na_align(sizeof(TypeTable));
  static constexpr size_t step = status + 256;
  static constexpr size_t mode = step + 256;
  static constexpr size_t sys_free = mode + 256;
  static constexpr size_t first = sys_free + 256;
  static constexpr size_t total = first + 256;
};

}  // namespace

// The scratch array (about 11 MB). In host code its name is only a stand-in
// for the device symbol; its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_forces_scratch[NaLayout::total];

namespace {

std::mutex g_na_mutex;
unsigned char* g_na_ptr[256] = {};  // per device: device address of g_forces_scratch

int na_fail(const std::string& m, int code = MD_ERR_INVALID_ARG) { return fail(nullptr, code, m); }

__global__ void k_na_load_x(int64_t n, const double* __restrict__ xa, double* __restrict__ x) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  x[i] = xa[3 * i];
  x[n + i] = xa[3 * i + 1];
  x[2 * n + i] = xa[3 * i + 2];
}

}  // namespace

extern "C" int md_forces_noalloc(const md_surface* surf, const md_params* prm, int64_t n, const double* d_x,
                                 const int32_t* d_type, const int32_t* d_mol, const uint8_t* d_constrained,
                                 double* d_f, double* d_u, void* cuda_stream) {
  if (!surf || !prm) return na_fail("surf and prm must not be NULL");
  if (n < 0 || n > kNaMaxParticles)
    return na_fail("md_forces_noalloc: n must be in [0, " + std::to_string(kNaMaxParticles) + "]");
  if (n > 0 && (!d_x || !d_f)) return na_fail("d_x and d_f must not be NULL");
  SysDev S;
  std::string why;
  if (check_system(*surf, *prm, S, why) != MD_OK) return na_fail("md_forces_noalloc: " + why);
  TypeTable T;
  fill_types(*prm, T);
  double rcmax = 0.0;
  for (int a = 0; a < prm->ntypes; ++a)
    for (int b = 0; b < prm->ntypes; ++b) rcmax = std::max(rcmax, prm->rcut[a][b]);
  const int has_pairs = rcmax > 0.0;
  const double rc_eff =
      (double)std::nextafter((float)(std::max(rcmax, prm->cell_size) * (1.0 + 1.0 / 4096.0)), INFINITY);
  uint64_t cells = 1;
  for (int d = 0; d < 3; ++d) {
    if (!has_pairs) {
      S.nc[d] = 1;
      S.cs[d] = 1.0;
      S.grid_lo[d] = 0.0;
    } else if (prm->periodic[d]) {
      const double L = prm->box_hi[d] - prm->box_lo[d];
      const int nc = (int)std::floor(L / rc_eff);
      if (nc < 3) return na_fail("a periodic axis must be at least 3 cells long");
      S.nc[d] = nc;
      S.cs[d] = L / nc;
      S.grid_lo[d] = prm->box_lo[d];
    } else {
      double lo, hi;
      if (prm->box_hi[d] > prm->box_lo[d]) {
        lo = prm->box_lo[d];
        hi = prm->box_hi[d];
      } else if (surface_extent(*surf, d, lo, hi)) {
        lo -= 2.0 * rc_eff;
        hi += 2.0 * rc_eff;
      } else {
        return na_fail("give box_lo/box_hi for an axis the surface does not bound");
      }
      const double ncd = std::ceil((hi - lo) / rc_eff);
      if (ncd > 1e6) return na_fail("cell grid too large along one axis");
      S.nc[d] = std::max(1, (int)ncd);
      S.cs[d] = rc_eff;
      S.grid_lo[d] = lo;
    }
    S.inv_cs[d] = 1.0 / S.cs[d];
    S.cs_f[d] = (float)S.cs[d];
    S.grid_lo_f[d] = (float)S.grid_lo[d];
    S.inv_cs_f[d] = (float)S.inv_cs[d];
    S.box_lo_f[d] = (float)S.box_lo[d];
    S.box_len_f[d] = (float)S.box_len[d];
    cells *= (uint64_t)S.nc[d];
  }
  if (cells >= 0xFFFFFFF0ull) return na_fail("more than 2^32 cells");
  S.slab = 0.0f;  // every stencil cell is visited
  S.cell_base = 0;
  S.first = 0;
  S.n = n;
  const int bonds = prm->beads_per_mol > 1, walls = prm->wall_enable != 0, excl = prm->exclude_intramol != 0;
  // device scratch address, once per device
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return na_fail("no current device", MD_ERR_NO_DEVICE);
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
      void* ptr = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&ptr, g_forces_scratch);
      if (e != cudaSuccess) return na_fail(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e), MD_ERR_CUDA);
      g_na_ptr[dev] = static_cast<unsigned char*>(ptr);
    }
    base = g_na_ptr[dev];
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  DevArrays A{};
  A.n = n;
  A.nsys = 1;
  A.pair_lanes = 1;
  if (cells <= kNaMaxBuckets) {
    A.hashed = 0;
    A.nbucket = (uint32_t)cells;
    A.log_t = 0;
  } else {
    A.hashed = 1;
    A.nbucket = kNaMaxBuckets;
    A.log_t = 18;
  }
  A.x = reinterpret_cast<double*>(base + NaLayout::x);
  A.f = base + NaLayout::f;
  A.rec = base + NaLayout::rec;
  A.rec_lo = prm->precision == MD_PREC_FP64 ? nullptr : reinterpret_cast<float4*>(base + NaLayout::rec_lo);
  A.ntypes = prm->ntypes;
  A.spin_limit = kDefaultSpinLimit;
  A.meta = reinterpret_cast<uint32_t*>(base + NaLayout::meta);
  A.mol = excl ? reinterpret_cast<int32_t*>(base + NaLayout::mol) : nullptr;
  A.cell = reinterpret_cast<uint32_t*>(base + NaLayout::cell);
  A.rank = reinterpret_cast<uint32_t*>(base + NaLayout::rank);
  A.count = reinterpret_cast<uint32_t*>(base + NaLayout::count);
  A.start = reinterpret_cast<uint32_t*>(base + NaLayout::start);
  A.blocksum = reinterpret_cast<uint32_t*>(base + NaLayout::blocksum);
  A.tile_state = reinterpret_cast<unsigned long long*>(base + NaLayout::tile_state);
  A.scan = reinterpret_cast<ScanCtl*>(base + NaLayout::scan);
  A.stag = reinterpret_cast<uint32_t*>(base + NaLayout::stag);
  A.stag_tmp = reinterpret_cast<uint32_t*>(base + NaLayout::stag_tmp);
  A.scell = reinterpret_cast<uint32_t*>(base + NaLayout::scell);
  A.sys = reinterpret_cast<const SysDev*>(base + NaLayout::sys);
  A.types = reinterpret_cast<const TypeTable*>(base + NaLayout::types);
  A.sys_free = reinterpret_cast<int32_t*>(base + NaLayout::sys_free);
  A.status = reinterpret_cast<uint32_t*>(base + NaLayout::status);
  A.step = reinterpret_cast<unsigned long long*>(base + NaLayout::step);
  A.mode = reinterpret_cast<int32_t*>(base + NaLayout::mode);
  int64_t* d_first = reinterpret_cast<int64_t*>(base + NaLayout::first);
  const int64_t zero64 = 0;
  const uint32_t nn32 = (uint32_t)n;
  // the array keeps the last call's contents: reset what must start at zero
  cudaError_t e = cudaMemcpyAsync(base + NaLayout::sys, &S, sizeof(SysDev), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(base + NaLayout::types, &T, sizeof(TypeTable), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_first, &zero64, sizeof(int64_t), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(A.start + A.nbucket, &nn32, sizeof(uint32_t), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(A.count, 0, sizeof(uint32_t) * A.nbucket, st);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(A.tile_state, 0,
                        sizeof(unsigned long long) * ((A.nbucket + kScanPerBlock - 1) / kScanPerBlock), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(A.scan, 0, sizeof(ScanCtl), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(base + NaLayout::status, 0, 3 * 256 + 256, st);
  if (e == cudaSuccess && n > 0) {
    k_na_load_x<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, d_x, A.x);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = launch_build_meta(A, d_first, 1, d_type, d_constrained, d_mol, 0, st);
  if (has_pairs) {
    if (e == cudaSuccess) e = launch_bin(A, prm->precision, st);
    if (e == cudaSuccess) e = launch_cells_after_bin(A, 0, st);
    if (e == cudaSuccess) e = launch_bucket_build(A, prm->precision, st);
  }
  if (e == cudaSuccess) e = launch_pair(A, prm->precision, has_pairs, bonds, walls, excl, st);
  if (e == cudaSuccess && prm->beads_per_mol > 2 && prm->angle_k != 0.0) e = launch_bend(A, prm->precision, st);
  if (e == cudaSuccess) e = launch_get_forces(A, prm->precision, d_f, d_u, st);
  uint32_t status = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&status, A.status, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return na_fail(std::string("md_forces_noalloc: ") + cudaGetErrorString(e), MD_ERR_CUDA);
  if (status & kFlagOutOfGrid) return na_fail("a particle is outside the cell grid", MD_ERR_OUT_OF_GRID);
  if (status & kFlagOffSurface) return na_fail("a type is outside [0, ntypes)");
  return MD_OK;
}
