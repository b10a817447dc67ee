// Host-side helpers shared by the single-simulation API and the server.
#pragma once

#include <cstddef>

#include "../../include/pycool.h"
#include "internal.cuh"

namespace pycool {

// Device memory layout of one simulation.
//   state     : [Background][SimDesc][phi buf 0][phi buf 1][pi buf 0][pi buf 1]
//   workspace : [ticket, fault word (256 B)][group tickets][block partials: ncta * kNQ
//               doubles][group partials: ngroups * kNQ doubles]; the counters
//               [0, off_partials) must be zero before a launch.
// Potentials given at run time (runtime_model.cu): fields of a registered
// model id (-1 if unknown), and one stage of such a simulation.
int runtime_model_nfields(int id);
cudaError_t launch_runtime_stage(const SimDesc& d, const LaunchTable& t, int grid, cudaStream_t s);
// The compiled potential of a runtime-model simulation at `phis` (V', V into
// the simulation's runtime scratch).
cudaError_t launch_runtime_potential(const SimDesc& d, const double* phis, cudaStream_t s);

struct Layout {
  Geometry geo;
  size_t field_bytes;
  size_t off_bg, off_desc, off_fields, state_bytes;
  size_t off_ticket, off_gticket, off_partials, off_gpartials, ws_bytes;
  size_t off_prows;   // single-simulation API: rows of the persistent kernel (0 = none)
  size_t off_punits;  // single-simulation API: the persistent kernel's unit table
  size_t off_rt;      // runtime potentials: drifted fields, V', V (0 = none)
  size_t off_mean;    // single-simulation API: partial sums of the split forms' initial means
};

// Workspace layout of a launch of `ncta` blocks (fills the off_* / ws_bytes fields).
void workspace_layout(int ncta, Layout& L);

int stage_table(int order, double* w);
int model_nfields(int model);
Layout layout_for(const pycool_config& c);
// layout_for() plus the persistent kernel's partial-sum rows in the workspace
// (what pycool_query_bytes reports and pycool_create uses).
Layout sim_layout(const pycool_config& c);
cudaError_t encode_persist_maps(const SimDesc& d, const PGeo& g, PParams& p);
cudaError_t launch_persist(const SimDesc& d, const PParams& p, int grid, cudaStream_t s, int* bps);
// The persistent kernel's parameters for a state and workspace laid out by
// sim_layout() (api.cu); *fits: one block per SM fits.
pycool_status persist_setup(const pycool_config& cfg, const SimDesc& hd, const Layout& L,
                            char* state, char* ws, cudaStream_t st, PParams& p, bool* fits);
pycool_status validate(const pycool_config* c);
void fill_desc(SimDesc& d, const pycool_config& c, const Layout& L, char* state, char* ws);
cudaError_t launch_sweep(const SimDesc& d, const LaunchTable& t, int grid, cudaStream_t s);
cudaError_t encode_tensor_maps(SimDesc& d);
cudaError_t launch_arm(Background* bg, long long nsweeps, cudaStream_t s);
void observables(const Background& b, const SimDesc& d, double mpl, double rho_r0,
                 double rho_m0, pycool_observables* out);
// Output-interval observables (observe.cu), at a synchronised state b.
cudaError_t launch_energy_fields(const SimDesc& d, const Background& b, double* rho, double* P,
                                 cudaStream_t s);
cudaError_t launch_field_values(const SimDesc& d, const Background& b, int which, int f,
                                double* out, cudaStream_t s);
cudaError_t launch_spectrum_bins(const void* spec, int n, const int32_t* order,
                                 const int32_t* start, int nbins, double* power, cudaStream_t s);
// Fault injection (pycool_debug_fail_alloc): true if this device allocation
// is to report failure (consumes one of the requested failures).
bool injected_alloc_failure();

}  // namespace pycool
