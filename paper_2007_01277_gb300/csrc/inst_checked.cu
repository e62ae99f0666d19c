// inst_checked.cu -- fused pairs compiled with checked barriers.
//
// The same bodies and the same 2-way kernel as the production instances,
// compiled with HF_CHECKED_BARRIERS: every interval barrier (the
// "bar.sync id, d_k" of Sec. 3.1) becomes a software barrier over the
// interval's warps whose wait is bounded by the global timer, so a barrier
// schedule that can never complete ends with kErrBarrierExpired in the
// device error word instead of a hang.  Everything from kernels.cuh is
// compiled into namespace hf_chk (the namespace name is redefined around the
// include), so these kernels are distinct symbols from the production ones;
// the registry entries share hfl::Instance.  Only pairs whose bodies have
// barriers are compiled, without a register bound.
#include <cstdint>
#include <cstring>
#include <utility>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../include/hfuse.h"
#include "hf_launch.h"

#define HF_CHECKED_BARRIERS 1
#define hf hf_chk
#include "kernels.cuh"
#undef hf

namespace hf_chk {
static const hfl::Instance kChecked[] = {
    make_pair_instance<BodyHist, BodyPhilox, 0>(),
    make_pair_instance<BodyBn, BodyHist, 0>(),
    make_pair_instance<BodyBn, BodyPoly, 0>(),
    make_pair_instance<BodyStreamTmpl, BodyStreamTmpl, 0>(),
};
} // namespace hf_chk

namespace hfl {
const Instance *checked_pair_table(int *n)
{
    *n = (int)(sizeof hf_chk::kChecked / sizeof hf_chk::kChecked[0]);
    return hf_chk::kChecked;
}
} // namespace hfl
