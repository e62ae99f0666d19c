// hf_launch.h -- host-side launch records shared by every compiled fused
// instance: the arguments of one 2-way launch and the registry entry of one
// instance.  They live outside the kernels' namespace so that instances
// compiled in another namespace (the checked-barrier build of
// inst_checked.cu) share one registry type with the production ones.
#pragma once
#include <cuda_runtime.h>

namespace hfl {

struct PairLaunch {
    const void *const *args;   // [0] body A args, [1] body B args
    int w_split, n_low, n_high;
    unsigned smem_high, smem_total;
    int low_is_a;
    int grid, d0;
    unsigned *err;
    unsigned ring_stage[2];   // low, high interval
    int ring_stages[2];
};

// Registry entry of one compiled instance.
struct Instance {
    int body_a, body_b;   // -1, -1 for the N-way kernel
    int regcap;           // 0 = none
    const void *func;     // the __global__ symbol
    cudaError_t (*launch_pair)(const PairLaunch &, cudaStream_t);
};

// The pairs compiled with bounded software barriers (inst_checked.cu).
const Instance *checked_pair_table(int *n);

} // namespace hfl
