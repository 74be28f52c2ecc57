// validate.h -- argument checks shared by the entry points that take a
// problem description (aderdg_create, aderdg_step_noalloc).
#pragma once
#include "aderdg.h"

namespace aderdg {

// Constants of the uniform material of Eq. 1's flux (aderdg_params::pde_const):
// nullptr if admissible, else the reason.  Acoustics needs a positive density
// and sound speed, Euler an adiabatic index above 1 (Sec. 7), elasticity a
// positive density and P-wave speed.
inline const char *check_pde_const(int pde, const double *c) {
  if (pde == ADERDG_ACOUSTICS && !(c[0] > 0 && c[1] > 0)) return "acoustics needs rho > 0 and c > 0";
  if (pde == ADERDG_EULER && !(c[0] > 1.0)) return "Euler needs gamma > 1";
  if (pde == ADERDG_ELASTICITY && !(c[0] > 0 && c[1] > 0)) return "elasticity needs rho > 0 and cp > 0";
  return nullptr;
}

// material_jumps of aderdg_params: nullptr if admissible, else the reason.
// The non-conservative form needs elasticity (the PDE with a per-cell
// material) in the fused form with the time-modal (line-owner) predictor.
inline const char *check_material_jumps(int value, int pde, int form, int predictor) {
  if (value != ADERDG_JUMPS_PER_CELL_FLUX && value != ADERDG_JUMPS_NONCONSERVATIVE) return "bad material_jumps";
  if (value == ADERDG_JUMPS_NONCONSERVATIVE &&
      (pde != ADERDG_ELASTICITY || form != ADERDG_FORM_FUSED || predictor != ADERDG_PREDICT_AUTO))
    return "non-conservative material jumps need ELASTICITY, the fused form and the time-modal predictor";
  return nullptr;
}

}  // namespace aderdg
