// staged_occ.cu -- FP32 tables: the analysis stage with per-occurrence
// marginals and occurrence maxima (staged.cuh).
#include "staged.cuh"

namespace are {

namespace {
template <int JP>
void go(const SimArgs &a, const TermsF32 &t, int num_sms, cudaStream_t s)
{
    if (a.off) staged::launch_staged_t<float, JP, false, true>(a, t, num_sms, s);
    else staged::launch_staged_t<float, JP, true, true>(a, t, num_sms, s);
}
}  // namespace

int launch_staged32_occ(const SimArgs &a, int jp, const TermsF32 &t, int num_sms, cudaStream_t s)
{
    if (a.n_trials <= 0) return 0;
    switch (jp) {
    case 8: go<8>(a, t, num_sms, s); return 1;
    case 16: go<16>(a, t, num_sms, s); return 1;
    case 32: go<32>(a, t, num_sms, s); return 1;
    }
    throw Error{ARE_EINVAL, "no FP32 staged kernel for table width " + std::to_string(jp)};
}

}  // namespace are
