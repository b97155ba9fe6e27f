// step_bf16.cu -- step kernels instantiated for precision P_BF16.
#include "launch_step.cuh"
QW_DEFINE_STEP_LAUNCHERS(qw::P_BF16, bf16)
