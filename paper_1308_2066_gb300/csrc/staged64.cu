// staged64.cu -- FP64 tables: the analysis stage with warp-compacted FP64
// work (staged.cuh), a tuning candidate of the FP64 analysis.
#include "staged.cuh"

namespace are {

namespace {
template <int JP>
void go(const SimArgs &a, const TermsF64 &t, int num_sms, cudaStream_t s)
{
    if (a.off) staged::launch_staged_t<double, JP, false>(a, t, num_sms, s);
    else staged::launch_staged_t<double, JP, true>(a, t, num_sms, s);
}
}  // namespace

int launch_staged64(const SimArgs &a, int jp, const TermsF64 &t, int num_sms, cudaStream_t s)
{
    if (a.n_trials <= 0) return 0;
    switch (jp) {
    case 4: go<4>(a, t, num_sms, s); return 1;
    case 8: go<8>(a, t, num_sms, s); return 1;
    case 12: go<12>(a, t, num_sms, s); return 1;
    case 16: go<16>(a, t, num_sms, s); return 1;
    case 20: go<20>(a, t, num_sms, s); return 1;
    case 24: go<24>(a, t, num_sms, s); return 1;
    case 28: go<28>(a, t, num_sms, s); return 1;
    case 32: go<32>(a, t, num_sms, s); return 1;
    }
    throw Error{ARE_EINVAL, "no FP64 staged kernel for table width " + std::to_string(jp)};
}

}  // namespace are
