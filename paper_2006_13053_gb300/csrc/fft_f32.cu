// FP32 instantiations of the Bluestein transforms (FP32 or FP64 input, FP32 output).
#include "bluestein.cuh"

namespace sfft {

int launch_bluestein_f32(bool in_double, const BlueJob* djobs, int njobs, int maxN, int mode, int sign, int epi,
                         const InstDesc* insts, cudaStream_t st, void* ob, const void* ab, int threads, int upair) {
    if (in_double) return launch_t<float, double, float>(djobs, njobs, maxN, mode, sign, epi, insts, st, ob, ab, threads, upair);
    return launch_t<float, float, float>(djobs, njobs, maxN, mode, sign, epi, insts, st, ob, ab, threads, upair);
}

}  // namespace sfft
