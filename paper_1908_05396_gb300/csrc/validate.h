// validate.h -- argument checks and parameter set-up shared by every entry
// point that takes a problem statement (clbm_create, clbm_collide_nodes,
// clbm_step_noalloc), so that a new clamp, rate or limit reaches all of them.
#pragma once

#include <cmath>
#include <string>

#include "../../include/clbm.h"
#include "launch.h"

namespace clbm {

// Largest grid extent in y and z of a CUDA launch: the step kernels launch
// one block row per z plane, so nz (and ny, with blocks one row high) must
// stay within it.
constexpr int MAX_GRID_YZ = 65535;

// Clamp defaults of the domain (0 selects them): rho0 = 1, nu in [5e-4, 10].
inline void domain_defaults(const clbm_domain* d, double* rho0, double* nu_min, double* nu_max) {
  *rho0 = d->rho0 > 0.0 ? d->rho0 : 1.0;
  *nu_min = d->nu_min > 0.0 ? d->nu_min : 5e-4;
  *nu_max = d->nu_max > 0.0 ? d->nu_max : 10.0;
}

// Physical parameters: K > 0 (the consistency coefficient of the power law),
// n in (0, 3], 0 < nu_min < nu_max < inf.
inline bool check_phys(double K, double n, double nu_min, double nu_max, std::string& why) {
  if (!(K > 0.0) || !std::isfinite(K)) { why = "K must be finite and > 0"; return false; }
  if (!(n > 0.0 && n <= 3.0)) { why = "n must lie in (0, 3]"; return false; }
  if (!(nu_min > 0.0 && nu_max > nu_min) || !std::isfinite(nu_max)) {
    why = "need 0 < nu_min < nu_max < inf";
    return false;
  }
  return true;
}

inline bool check_force(const double* F, std::string& why) {
  if (F)
    for (int a = 0; a < 3; ++a)
      if (!std::isfinite(F[a])) { why = "non-finite force"; return false; }
  return true;
}

// Dimensions, face kinds, periodic pairs and the lid; U receives U_lid (0
// where NULL).  A LID face needs a lid velocity below the Mach limit 0.3,
// tangential to every LID face.
inline bool check_domain(const clbm_domain* d, const double* U_lid, double U[3],
                         std::string& why) {
  if (d->nx < 1 || d->ny < 1 || d->nz < 1) {
    why = "lattice dimensions must be >= 1";
    return false;
  }
  if (d->ny > MAX_GRID_YZ || d->nz > MAX_GRID_YZ) {
    why = "ny and nz must be <= 65535 (one launch grid row per y row and z plane)";
    return false;
  }
  bool has_lid = false;
  for (int f = 0; f < 6; ++f) {
    if (d->face[f] < CLBM_PERIODIC || d->face[f] > CLBM_LID) {
      why = "unknown face kind";
      return false;
    }
    has_lid = has_lid || d->face[f] == CLBM_LID;
  }
  for (int a = 0; a < 3; ++a)
    if ((d->face[2 * a] == CLBM_PERIODIC) != (d->face[2 * a + 1] == CLBM_PERIODIC)) {
      why = "a periodic face needs a periodic opposite face";
      return false;
    }
  for (int a = 0; a < 3; ++a) U[a] = U_lid ? U_lid[a] : 0.0;
  if (has_lid) {
    if (!U_lid) { why = "LID face without U_lid"; return false; }
    const double mag = std::sqrt(U[0] * U[0] + U[1] * U[1] + U[2] * U[2]);
    if (!(mag < 0.3)) { why = "|U_lid| must be < 0.3"; return false; }
    for (int f = 0; f < 6; ++f)
      if (d->face[f] == CLBM_LID && U[f / 2] != 0.0) {
        why = "U_lid must be tangential to every LID face";
        return false;
      }
  }
  return true;
}

// PhysParams of a checked problem statement, relaxation rates omega_9..18 = 1.
inline void fill_params(PhysParams& P, double K, double n, const double* F, double rho0,
                        double nu_min, double nu_max, clbm_dtype dtype) {
  P.rho0 = rho0;
  for (int a = 0; a < 3; ++a) P.F[a] = F ? F[a] : 0.0;
  P.has_force = (P.F[0] != 0.0 || P.F[1] != 0.0 || P.F[2] != 0.0) ? 1 : 0;
  P.K = K;
  P.logK3 = std::log(3.0 * K);
  P.n = n;
  P.newtonian = (n == 1.0) ? 1 : 0;
  P.nu_min = nu_min;
  P.nu_max = nu_max;
  P.ylo = std::log(3.0 * nu_min);
  P.yhi = std::log(3.0 * nu_max);
  P.inv_scale = (dtype == CLBM_F16S || dtype == CLBM_F16R) ? 1.0 / F16_SCALE : 1.0;
}

}  // namespace clbm
