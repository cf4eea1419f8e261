// Physics step, 128 threads per environment (the common case: up to a few
// dozen bodies, seven environments resident per SM).  The kernels and their
// launchers are in physics_impl.cuh.
#define VUDA_SIM_THREADS 128
#define VUDA_SIM_NS_BEGIN
#define VUDA_SIM_NS_END
#include "physics_impl.cuh"
