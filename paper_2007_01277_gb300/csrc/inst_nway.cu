// inst_nway.cu -- the N-way persistent fused kernel (all bodies behind a
// runtime switch, one instance per register cap) and the standalone kernels.
#include "kernels.cuh"

namespace hf {

// Without an explicit cap the N-way kernel is still bounded so that a
// 512-thread block always fits (at most 128 registers per thread).
__global__ void __launch_bounds__(512) k_nway(const __grid_constant__ NwayParams p) { nway_body(p); }

#define HF_NWAY_ENTRY(R) Instance{-1, -1, R, reinterpret_cast<const void *>(&k_nway_cap<R>), nullptr},
static const Instance kNway[] = {
    Instance{-1, -1, 0, reinterpret_cast<const void *>(&k_nway), nullptr},
    HF_REGCAP_LIST(HF_NWAY_ENTRY)};

const Instance *nway_table(int *n)
{
    *n = (int)(sizeof kNway / sizeof kNway[0]);
    return kNway;
}

template <class B>
SingleEntry make_single()
{
    return SingleEntry{B::kId, reinterpret_cast<const void *>(&k_single<B>), &launch_single<B>};
}

static const SingleEntry kSingles[] = {
    make_single<BodyBn>(),   make_single<BodyUpsample>(), make_single<BodyMaxpool>(),
    make_single<BodyIm2col>(), make_single<BodyHist>(),   make_single<BodyPhilox>(),
    make_single<BodyPoly>(), make_single<BodyBf16Axpy>(), make_single<BodyStreamTmpl>(),
    make_single<BodySha256d>(), make_single<BodyBlake256>(), make_single<BodyBlake2b>()};

const SingleEntry *single_table(int *n)
{
    *n = (int)(sizeof kSingles / sizeof kSingles[0]);
    return kSingles;
}

} // namespace hf
