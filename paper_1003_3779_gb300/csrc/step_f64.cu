// step_f64.cu -- step kernels instantiated for precision P_F64.
#include "launch_step.cuh"
QW_DEFINE_STEP_LAUNCHERS(qw::P_F64, f64)
