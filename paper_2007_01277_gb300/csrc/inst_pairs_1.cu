// inst_pairs_1.cu -- compiled 2-way fused instances, one per (body A,
// body B, register cap); cap 0 means no register bound.
#include "kernels.cuh"

namespace hf {

#define HF_CAP_ENTRY(R) make_pair_instance<A_, B_, R>(),
static const Instance kTable[] = {
#define A_ BodyStreamTmpl
#define B_ BodyStreamTmpl
    make_pair_instance<A_, B_, 0>(), HF_REGCAP_LIST(HF_CAP_ENTRY)
#undef A_
#undef B_
#define A_ BodyBn
#define B_ BodyUpsample
    make_pair_instance<A_, B_, 0>(), HF_REGCAP_LIST(HF_CAP_ENTRY)
#undef A_
#undef B_
#define A_ BodyBn
#define B_ BodyHist
    make_pair_instance<A_, B_, 0>(), HF_REGCAP_LIST(HF_CAP_ENTRY)
#undef A_
#undef B_
#define A_ BodyBn
#define B_ BodyIm2col
    make_pair_instance<A_, B_, 0>(), HF_REGCAP_LIST(HF_CAP_ENTRY)
#undef A_
#undef B_
};

const Instance *pair_table_1(int *n)
{
    *n = (int)(sizeof kTable / sizeof kTable[0]);
    return kTable;
}

} // namespace hf
