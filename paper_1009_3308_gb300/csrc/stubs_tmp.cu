// temporary: entry points still being written
#include "internal.h"
extern "C" {
int sphnse_state_init(sphnse_plan*, sphnse_state*, double, double, const double*) { return SPHNSE_E_UNSUPPORTED; }
int sphnse_step(sphnse_plan*, sphnse_state*, const double*, sphnse_step_info*) { return SPHNSE_E_UNSUPPORTED; }
int sphnse_replay_step(sphnse_plan*, sphnse_state*, const double*, double, int, int, sphnse_step_info*) { return SPHNSE_E_UNSUPPORTED; }
int sphnse_rhs_adjoint(sphnse_plan*, const double*, const double*, double*, double*) { return SPHNSE_E_UNSUPPORTED; }
int sphnse_adjoint_step(sphnse_plan*, double, int, double, const double*, double*, double*, double*) { return SPHNSE_E_UNSUPPORTED; }
int sphnse_adjoint_init(sphnse_plan*, double, const double*, double*, const double*, double*) { return SPHNSE_E_UNSUPPORTED; }
int sphnse_objective(sphnse_plan*, const double*, const double*, double, double, double*, double*) { return SPHNSE_E_UNSUPPORTED; }
}
