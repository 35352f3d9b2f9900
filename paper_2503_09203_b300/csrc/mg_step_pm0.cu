// Step-kernel instantiations whose physical parameters are class constants
// (PM = 0): every thruster count, variant and table source.
#include "mg_step.cuh"

namespace mg {

cudaError_t launch_step_pm0(const StepArgs& a, const ClassK* kc, const ClassG* kg, int nt, int var, int grid,
                            bool dependent, bool shared_sm, cudaStream_t st) {
  return launch_step_pm<0>(a, kc, kg, nt, var, grid, dependent, shared_sm, st);
}

cudaError_t prepare_tick_pm0(int nt, int var) { return prepare_tick_pm<0>(nt, var); }

cudaError_t occupancy_pm0(int nt, int var, bool kp, bool track, int* blocks_per_sm) {
  return occupancy_pm<0>(nt, var, kp, track, blocks_per_sm);
}

}  // namespace mg
