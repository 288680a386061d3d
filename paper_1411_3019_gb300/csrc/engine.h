// engine.h -- host-side launchers of the surfmd kernels (kernels.cu) used by
// the C ABI (capi.cu).
#pragma once

#include <cuda_runtime.h>

#include "surfmd.cuh"

namespace surfmd {

constexpr int kScanPerBlock = 8192;  // bucket counters scanned by one CTA

// Build the meta word of every particle (type, constrained bit, system id)
// and the molecule ids. type/con/mol may be null (defaults of md_set_state).
cudaError_t launch_build_meta(const DevArrays& A, const int64_t* d_first, int nsys,
                              const int32_t* d_type, const uint8_t* d_con, const int32_t* d_mol,
                              int has_mol_default, cudaStream_t st);

// x, v ([n][3] device) -> SoA state; validate g, project v, p = m v.
cudaError_t launch_set_state(const DevArrays& A, const double* d_x_aos, const double* d_v_aos,
                             cudaStream_t st);

// x, p_half ([n][3] device) -> SoA state (checkpoint restore).
cudaError_t launch_restore(const DevArrays& A, const double* d_x_aos, const double* d_ph_aos,
                           cudaStream_t st);

// Cell list of the current positions: bin, scan, scatter, canonical sort.
// `advance` = 1 also moves the step counter on by one (inside md_step).
cudaError_t launch_bin(const DevArrays& A, int precision, cudaStream_t st);
cudaError_t launch_bucket_build(const DevArrays& A, int precision, cudaStream_t st);
cudaError_t launch_cells_after_bin(const DevArrays& A, int advance, cudaStream_t st);
cudaError_t launch_scan(const DevArrays& A, int advance, cudaStream_t st);
// Visiting order of the pair kernel: counting sort of the particles by
// (system << sys_shift) | (Morton code of (cell coords >> coord_shift)) >>
// morton_drop. O holds the key counters, starts and scan state (its nbucket =
// number of keys); A.rank is reused as scratch (call it after the cell list
// is complete, before the next binning).
cudaError_t launch_order(const DevArrays& A, const DevArrays& O, uint32_t coord_shift, uint32_t morton_drop,
                         uint32_t sys_shift, uint32_t* order, cudaStream_t st);
cudaError_t launch_scatter(const DevArrays& A, cudaStream_t st);

// Conservative forces at the current positions into A.f.
// Neighbour-list build (only when *A.nl_dirty; every pair within r_c + skin).
cudaError_t launch_nl_build(const DevArrays& A, int precision, int excl, cudaStream_t st);
// Fused rebuild of the Verlet-list step (cooperative launch of `blocks` CTAs of
// 256 threads; rebuild_blocks gives the count, 0 if it cannot be launched):
// returns at once unless the rebuild flag is up, advances the step counter.
int rebuild_blocks(int precision, int excl, int64_t n);
cudaError_t launch_rebuild(const DevArrays& A, int precision, int excl, int blocks, cudaStream_t st);
cudaError_t launch_pair(const DevArrays& A, int precision, int has_pairs, int bonds, int walls,
                        int excl, cudaStream_t st);

// Combine + momentum half + position half (+ binning when has_pairs).
// Bend-angle forces added to the pair kernel's output (systems with angles).
cudaError_t launch_bend(const DevArrays& A, int precision, cudaStream_t st);
cudaError_t launch_integrate(const DevArrays& A, int precision, int has_pairs, cudaStream_t st);

// Step counter on by one, mode = 1 (used when there is no cell list).
cudaError_t launch_advance(const DevArrays& A, cudaStream_t st);

// p^k into A.pk from the state and A.f (momentum half only).
cudaError_t launch_finish(const DevArrays& A, int precision, cudaStream_t st);

// SoA -> [n][3] for x, v = p^k / m and p^{k-1/2}; outputs may be null.
cudaError_t launch_get_state(const DevArrays& A, double* d_x_aos, double* d_v_aos, double* d_ph_aos,
                             cudaStream_t st);

// Forces A.f -> [n][3] float64 and per-particle energies.
cudaError_t launch_get_forces(const DevArrays& A, int precision, double* d_f_aos, double* d_u,
                              cudaStream_t st);

// Resident engine: every system of J advances J.nsteps steps inside one
// launch (one CTA per system at a time, cell list and forces in shared
// memory); the step counter is advanced afterwards by launch_advance_n.
// threads: CTA size (a multiple of 32, <= kResidentMaxThreads); grid_cap > 0
// limits the CTAs.
size_t resident_smem_bytes(int precision, uint32_t nmax, uint32_t tmax);
cudaError_t launch_resident(const DevArrays& A, int precision, const ResidentJob& J, int bonds, int walls, int excl,
                            int threads, int grid_cap, cudaStream_t st);
cudaError_t launch_advance_n(const DevArrays& A, int32_t nsteps, cudaStream_t st);
// CTAs of the resident kernel that fit on one SM (0: none).
int resident_blocks_per_sm(int precision, int bonds, int walls, int excl, uint32_t nmax, uint32_t tmax, int threads);

// out_f[i] = in[i] rounded to float32, out_d[i] = out_f[i] widened to float64,
// by the integer-pipe conversions of the mixed path.
cudaError_t launch_check_conversions(const double* in, int64_t n, float* out_f, double* out_d, cudaStream_t st);

// Peak probe: blocks x 256 threads, each 8 independent FMA chains of iters
// steps, in float64 (precision 0) or float32 (1).
cudaError_t launch_fma_probe(int precision, int blocks, int iters, cudaStream_t st);

// Residuals: out[0] = max |g|/|grad g|, out[1] = max |g|, out[2] = max |n.v|/|n|
// (stored as the bit patterns of non-negative doubles; zeroed inside).
cudaError_t launch_residual(const DevArrays& A, unsigned long long* d_out, cudaStream_t st);

// Per-system sums: 8 doubles per system (K, U, msd, r0.rt/R^2, ndof, max g/|n|,
// max |n.v|/|n|, n), zeroed inside.
cudaError_t launch_observables(const DevArrays& A, int precision, double* d_obs, cudaStream_t st);

}  // namespace surfmd
