// fft_plan.h -- the radix plan of one FFT length (host and device code).
#pragma once

namespace svh {

constexpr int MAX_STAGES = 16;

// N = R[0] * R[1] * ... * R[nst - 1], stages applied in that order
struct FftPlan {
    int N;
    int nst;
    int R[MAX_STAGES];
};

}  // namespace svh
