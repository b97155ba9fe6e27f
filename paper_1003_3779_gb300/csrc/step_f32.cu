// step_f32.cu -- step kernels instantiated for precision P_F32.
#include "launch_step.cuh"
QW_DEFINE_STEP_LAUNCHERS(qw::P_F32, f32)
