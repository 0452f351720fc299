// Host-side helpers shared by the single-grid context (api.cu) and the batch
// driver (batch.cu): validation, nonlinear-term tables, operator coefficients,
// Chebyshev weights and the process-wide measurement state.
#pragma once

#include <string>
#include <vector>

#include "apfc_internal.cuh"

namespace apfc {

// lattice and parameters of Sec. II (k_j finite, hex: J = 3 in 2D with sum k_j = 0,
// bcc: J = 6 in 3D, Bx > 0)
bool valid_problem(const apfc_lattice& lat, const apfc_params& p);
bool valid_opts(const apfc_opts& o, std::string& err);

// <n^p> resonance tables of the nonlinear term and the energy (Sec. II.A)
bool build_tables(const apfc_lattice& L, const apfc_params& P, NonlinTable& nt, EnergyTable& et, std::string& err);

// Operator coefficients of the block system for a time step dt on grid (n, h).
// make_coef_into returns nullptr on success, else a static message; it
// allocates nothing.
const char* make_coef_into(const apfc_lattice& lat, const apfc_params& par, const apfc_grid& grid, int tau_mode,
                           double dt, OpCoef& o);
bool make_coef(const apfc_lattice& lat, const apfc_params& par, const apfc_grid& grid, int tau_mode, double dt,
               OpCoef& o, std::string& err);

// Chebyshev recurrence weights for m applications of D (Saad, Sec. 12.3); they
// depend on the spacing only, not on the grid size.  cheb_weights_into fills
// max(m, 1) entries of w (zeroed first) and allocates nothing.
std::vector<ChebStep> cheb_weights_for(const OpCoef& c, const apfc_grid& grid, int m);
void cheb_weights_into(const OpCoef& c, const apfc_grid& grid, int m, ChebStep* w);

// Relative tolerance of the next FP32 inner solve of one amplitude in iterative
// refinement: 2 (stop at once) if its outer residual already meets tol; otherwise
// just enough to bring the outer residual to a quarter of tol, never tighter than
// tol_inner nor looser than 1/2.
double inner_tol(double tol, double tol_inner, double rnorm2, double bnorm2);

// Measurement (see apfc_profile_start): dev receives the device byte counters.
bool profiler_start(cudaStream_t s, int timed_id, unsigned long long** dev, std::string& err);
bool profiler_read(cudaStream_t s, int id, double* ms, long long* launches, double* bytes, long long* all_launches,
                   std::string& err);
void profiler_stop();
bool profiler_on();

}  // namespace apfc
