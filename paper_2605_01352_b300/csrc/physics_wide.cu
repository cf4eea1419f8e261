// Physics step, 512 threads per environment: for environments of more than
// 64 bodies, whose pair and contact phases have work for that many threads
// and whose shared memory leaves room for only one or two environments per
// SM.  Same kernels as physics.cu (physics_impl.cuh), launchers in
// namespace vuda::wide.
#define VUDA_SIM_THREADS 512
#define VUDA_SIM_NS_BEGIN namespace wide {
#define VUDA_SIM_NS_END }
#include "physics_impl.cuh"
