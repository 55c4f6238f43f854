// FP64 instantiation of the Bluestein transforms.
#include "bluestein.cuh"

namespace sfft {

int launch_bluestein_f64(const BlueJob* djobs, int njobs, int maxN, int mode, int sign, int epi, const InstDesc* insts,
                         cudaStream_t st, void* ob, const void* ab, int threads, int upair) {
    return launch_t<double, double, double>(djobs, njobs, maxN, mode, sign, epi, insts, st, ob, ab, threads, upair);
}

}  // namespace sfft
