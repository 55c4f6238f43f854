// Double-float instantiation of the Bluestein transforms (FP32 input, high words out, low words
// to the job's aux buffer).
#include "bluestein.cuh"

namespace sfft {

int launch_bluestein_df64(const BlueJob* djobs, int njobs, int maxN, int mode, int sign, int epi, const InstDesc* insts,
                         cudaStream_t st, void* ob, const void* ab, int threads, int upair) {
    return launch_t<df64, float, float>(djobs, njobs, maxN, mode, sign, epi, insts, st, ob, ab, threads, upair);
}

}  // namespace sfft
