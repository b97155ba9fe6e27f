// step_comp.cu -- step kernels instantiated for precision P_COMP.
#include "launch_step.cuh"
QW_DEFINE_STEP_LAUNCHERS(qw::P_COMP, comp)
