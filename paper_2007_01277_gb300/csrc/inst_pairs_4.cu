// inst_pairs_4.cu -- compiled 2-way fused instances of the three hash
// kernels (the compute+compute pairs of Sec. 4.2), one per register cap;
// cap 0 means no register bound.
#include "kernels.cuh"

namespace hf {

#define HF_CAP_ENTRY(R) make_pair_instance<A_, B_, R>(),
static const Instance kTable[] = {
#define A_ BodySha256d
#define B_ BodyBlake256
    make_pair_instance<A_, B_, 0>(), HF_REGCAP_LIST(HF_CAP_ENTRY)
#undef A_
#undef B_
#define A_ BodySha256d
#define B_ BodyBlake2b
    make_pair_instance<A_, B_, 0>(), HF_REGCAP_LIST(HF_CAP_ENTRY)
#undef A_
#undef B_
#define A_ BodyBlake256
#define B_ BodyBlake2b
    make_pair_instance<A_, B_, 0>(), HF_REGCAP_LIST(HF_CAP_ENTRY)
#undef A_
#undef B_
};

const Instance *pair_table_4(int *n)
{
    *n = (int)(sizeof kTable / sizeof kTable[0]);
    return kTable;
}

} // namespace hf
