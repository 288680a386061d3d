// surfmd.cuh -- device-side types and helpers of the constrained Langevin
// step (Paquay & Kusters, Algorithm 1 and Algorithm S1) on sm_103a.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace surfmd {

constexpr int kMaxTypes = 8;

// Bits of the device status word (match MD_FLAG_* of md.h).
constexpr uint32_t kFlagRattle = 0x1u;
constexpr uint32_t kFlagNonfinite = 0x2u;
constexpr uint32_t kFlagOutOfGrid = 0x4u;
constexpr uint32_t kFlagTimeout = 0x8u;
constexpr uint32_t kFlagNlistFull = 0x10u;  // a particle had more neighbours than the list holds
constexpr uint32_t kFlagOffSurface = 0x100u;  // set-state validation only

enum SurfKind : int32_t {
  kNone = 0, kPlane = 1, kSphere = 2, kEllipsoid = 3, kTorus = 4, kBump = 5, kCylinder = 6, kXY2D = 7, kThylakoid = 8
};

// Per-particle meta word: type (bits 0-2), constrained (bit 3), system (bits 4-31).
__host__ __device__ inline uint32_t meta_pack(uint32_t type, uint32_t con, uint32_t sys) {
  return (type & 7u) | ((con & 1u) << 3) | (sys << 4);
}
__host__ __device__ inline uint32_t meta_type(uint32_t m) { return m & 7u; }
__host__ __device__ inline bool meta_con(uint32_t m) { return (m >> 3) & 1u; }
__host__ __device__ inline uint32_t meta_sys(uint32_t m) { return m >> 4; }

// A double-float value h + l (two float32 numbers, |l| <= ulp(h) / 2); the
// arithmetic is in df.cuh.
struct DF {
  float h, l;
};

// One system's constants as the kernels read them.
struct SysDev {
  // surface g(x) = 0
  int32_t kind;
  int32_t axis;              // cylinder axis
  double c[3];               // centre / plane point
  double p[4];               // shape parameters
  double inv_a2[3];          // ellipsoid 1/a_d^2
  float c_f[3], p_f[4], inv_a2_f[3];  // float32 copies for surface directions
  // integration
  double dt, half_dt, kT, gamma;
  double comb;               // 1 / (1 + gamma dt / 2)
  double noise_unit;         // sqrt(2 kT gamma / dt); times sqrt(m) per particle
  double tol, tol2;           // RATTLE tolerance and its square
  float gamma_f, comb_f, noise_unit_f;
  int32_t max_newton, frozen;
  // per particle type: dt/m and m/dt (float64), dt/m (float32)
  double dtm[kMaxTypes], inv_dtm[kMaxTypes];
  float dtm_f[kMaxTypes];
  float half_dt_f, tol_f;
  double gconst;             // constant term of g: -R^2 (sphere, cylinder), -r^2 (torus)
  // double-float copies for the mixed path's position half
  DF c_df[3], inv_a2_df[3], pn_df[3];  // centre, ellipsoid 1/a_d^2, plane normal
  DF gconst_df, R_df;                  // constant term of g; torus R
  DF dt_df, half_dt_df;
  DF dtm_df[kMaxTypes], inv_dtm_df[kMaxTypes];  // dt/m and m/dt per type
  int32_t c_zero;            // 1: the centre is the origin
  int32_t pad_df;
  // box and cell grid
  double box_lo[3], box_len[3], inv_box_len[3];
  int32_t periodic[3];
  int32_t pad0;
  double grid_lo[3], cs[3], inv_cs[3];
  float cs_f[3];
  float grid_lo_f[3], inv_cs_f[3], box_lo_f[3], box_len_f[3];  // float32 binning
  float slab;                // tangent-slab half thickness for stencil pruning (0: off)
  int32_t nc[3];
  uint32_t cell_base;
  // resident engine: this system's buckets in shared memory (res_t of them,
  // res_t = 2^res_log_t; hashed when the grid has more cells than that)
  uint32_t res_t;
  int32_t res_log_t, res_hashed;
  // bonds, exclusions, walls
  int32_t bpm;
  int32_t excl;
  double bond_k, bond_r0;
  int32_t wall;
  int32_t pad1;
  double wall_lo, wall_hi, wall_eps, wall_sigma, wall_rc;
  // capsid-model terms: bend angles, type-dependent bond lengths, spherical wall
  double angle_k, angle_theta0;
  double angle_sin0, angle_cos0;  // sin and cos of theta0
  int32_t bond_mix, wall_kind;
  double wall_radius, wall_center[3];
  // noise key, particle range
  uint32_t seed_lo, replica;
  int64_t first, n;
};

// Pair tables shared by all systems of a handle (symmetric).
struct TypeTable {
  double eps[kMaxTypes][kMaxTypes];
  double sig2[kMaxTypes][kMaxTypes];
  double rc2[kMaxTypes][kMaxTypes];
  double shift[kMaxTypes][kMaxTypes];  // phi(r_c)
  double lin[kMaxTypes][kMaxTypes];    // phi'(r_c) for the linearly smoothed form, else 0
  double rc[kMaxTypes][kMaxTypes];
  float eps_f[kMaxTypes][kMaxTypes];
  float sig2_f[kMaxTypes][kMaxTypes];
  float rc2_f[kMaxTypes][kMaxTypes];
  float shift_f[kMaxTypes][kMaxTypes];
  float lin_f[kMaxTypes][kMaxTypes];
  float rc_f[kMaxTypes][kMaxTypes];
  double bond_r0_mix[kMaxTypes][kMaxTypes];  // 2^(1/6) sigma_ij / 2
  double mass[kMaxTypes], inv_mass[kMaxTypes], sqrt_mass[kMaxTypes];
  float sqrt_mass_f[kMaxTypes];
  // mixed path, pair terms from double-float displacements (kernels.cu, lj_term_acc)
  float rc2m_f[kMaxTypes][kMaxTypes];  // screen: r_c^2 (1 + 2^-18) in float32
  DF rc2_df[kMaxTypes][kMaxTypes];     // r_c^2
  DF s6x2_df[kMaxTypes][kMaxTypes];    // 2 sigma^6
  float c24_f[kMaxTypes][kMaxTypes];   // 24 eps sigma^6
  float c4_f[kMaxTypes][kMaxTypes];    // 4 eps sigma^6
  float s6_f[kMaxTypes][kMaxTypes];    // sigma^6
};

template <typename R> struct V4;
template <> struct V4<float> { using T = float4; };
template <> struct V4<double> { using T = double4_32a; };

// Control words of the one-pass scan (zero at creation).
constexpr int kResidentMaxThreads = 512;  // CTA size limit of the resident kernel (64 registers at 2 CTAs)

// Work list of the resident engine: systems in the order CTAs take them
// (largest first), a queue counter (zero before the launch), steps per launch
// and the shared-memory capacity of one CTA.
struct ResidentJob {
  const int32_t* order;
  uint32_t* next;
  int32_t nsys, nsteps;
  uint32_t nmax, tmax;
};

// Grid barrier of the fused rebuild kernel (zero at creation): arrivals and
// the generation the waiting CTAs watch.
struct GridBar {
  uint32_t count;
  uint32_t gen;
};
constexpr int kRebuildMaxBlocks = 4096;  // CTAs of the fused rebuild kernel at most

struct ScanCtl {
  uint32_t tile;   // next tile index
  uint32_t done;   // tiles finished in this launch
  uint32_t epoch;  // launch counter tagging the tile states
  uint32_t pad;
};

// Arrays of one handle, passed by value to the kernels.
struct DevArrays {
  int64_t n;            // particles
  int32_t nsys;
  uint32_t nbucket;     // T
  int32_t hashed;       // 0: bucket = cell id; 1: hashed buckets
  int32_t log_t;
  int32_t pair_lanes;   // lanes per particle in the pair kernel (1, 2, 4 or 8)
  int32_t pair_tile;    // 0, or particles per warp (8, 16, 32) of the cell-tiled pair kernel (needs hashed == 0)
  int32_t pair_queue;   // mixed path with the Verlet list: 1 = warp-queued list walk (k_pair_nlq), 0 = per-lane walk
  int32_t list_warp;    // particles per warp of the warp-queued list walk (8, 16 or 32)
  // Verlet neighbour list (nl_dirty == null: off). Built from the cell list
  // with every pair within r_c + skin; between builds the integrator moves
  // the records in place and raises *nl_dirty when a particle has moved more
  // than skin / 2, and the cell list and the list are rebuilt in that step.
  uint32_t* nl_dirty;   // device flag: 1 = rebuild the cell list and the neighbour list
  uint32_t* nl;         // [n][nl_max] build scratch: entries by sorted slot, slot << 5 | stencil cell (0..26)
  uint32_t* nl_cnt;     // [n] entries per sorted slot
  // the lists packed by groups of 32 consecutive slots: group g = s & ~31 owns
  // entries [g nl_max, (g + 32) nl_max), its slots' lists one after another
  // in slot order, slot s's from nl_off[s]; the walks read these (nl is the
  // build's scratch)
  uint32_t* nl_pk;
  uint32_t* nl_off;     // [n] start of a slot's entries within its group's run
  uint32_t* smeta;      // [n] meta of each sorted slot (written with the records at a rebuild), or null
  // mixed path with the list: the unit normals xi^k of the last integrated
  // step k (by particle; the next step's force combination needs them again)
  // and that step, ~0 when none is stored (after a state is set)
  float4* noise;
  unsigned long long* noise_k;
  int32_t store_noise;  // 1: store and reuse the normals (MD_OPT_STORE_NOISE), 0: draw both steps' again
  void* rec0;           // [n] records at the last build, by particle
  double* xb;           // [3][n] positions at the last build (user order)
  unsigned long long* nl_builds;  // list builds so far (counter)
  int32_t nl_max;
  float nl_half_skin2;  // (skin / 2)^2
  double nl_skin;
  int32_t rec_cell;     // 1: a record's w word holds type | cell << 3 (no exclusions,
                        // cells < 2^29), so the pair kernel needs no sorted-cell load;
                        // 0: type | molecule << 3
  double* x;            // [3][n] positions (unwrapped), SoA
  double* ph;           // [3][n] p^{k-1/2} (or p^k before the first step)
  double* pk;           // [3][n] p^k scratch
  double* xref;         // [3][n] MSD reference
  void* f;              // [n] float4 / double4_32a: conservative force + energy
  uint32_t* meta;       // [n]
  int32_t* mol;         // [n] molecule ids (exclusions) or null
  uint32_t* cell;       // [n] cell id of each particle
  uint32_t* rank;       // [n] rank inside its bucket (atomic order)
  uint32_t* count;      // [T] bucket occupancy
  uint32_t* start;      // [T+1] bucket start
  uint32_t* blocksum;   // [scan blocks] (unused by the one-pass scan)
  unsigned long long* tile_state;  // [scan blocks] published tile aggregates / prefixes
  ScanCtl* scan;        // one-pass scan control words
  uint32_t* slot_of;    // [n] particle -> its sorted slot (written with the records)
  const uint32_t* order;  // [n] visiting order of the pair kernel (spatially coherent) or null
  uint32_t* stag;       // [n] sorted slot -> particle (canonical order)
  uint32_t* stag_tmp;   // [n] slot -> particle in atomic order (before the canonical sort)
  uint32_t* scell;      // [n] sorted slot -> cell id
  void* rec;            // [n] float4 / double4_32a cell-relative offsets + type/mol bits
  float4* rec_lo;       // [n] mixed path: offset - record (the low parts; w unused), else null
  float4* rec0_lo;      // [n] mixed path with the neighbour list: rec_lo at the last build, by particle
  int32_t ntypes;       // particle types in use (a type must lie in [0, ntypes))
  uint32_t spin_limit;  // reads of a predecessor's scan word before the wait gives up
  GridBar* gbar;        // fused rebuild: grid barrier
  uint32_t* rb_sum;     // fused rebuild: [kRebuildMaxBlocks] bucket-counter sums of the CTAs' ranges
  const SysDev* sys;    // [nsys]
  const TypeTable* types;  // pair and mass tables shared by the systems
  int32_t* sys_free;    // [nsys] unconstrained particles per system (set with the state)
  uint32_t* status;     // device status word
  unsigned long long* step;  // device step counter k
  int32_t* mode;        // 0: state holds p^k (first step pending); 1: holds p^{k-1/2}
};

}  // namespace surfmd
