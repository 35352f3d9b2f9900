// Step-kernel instantiations whose physical parameters are per-env parameter planes with the payload
// (PM = 2): every thruster count, variant and table source.
#include "mg_step.cuh"

namespace mg {

cudaError_t launch_step_pm2(const StepArgs& a, const ClassK* kc, const ClassG* kg, int nt, int var, int grid,
                            bool dependent, bool shared_sm, cudaStream_t st) {
  return launch_step_pm<2>(a, kc, kg, nt, var, grid, dependent, shared_sm, st);
}

cudaError_t occupancy_pm2(int nt, int var, bool kp, bool track, int* blocks_per_sm) {
  return occupancy_pm<2>(nt, var, kp, track, blocks_per_sm);
}

}  // namespace mg
