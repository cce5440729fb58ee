// Decoding with float message storage: the launch sequences of
// decode_run.cuh and the kernels they use, for every slab width.
#include "decode_run.cuh"

namespace mld {

int run_decode_f32(mld_decoder *d, const float *in, const float *sigma, const uint8_t *syn, int32_t batch,
                     int32_t iters, bool et, uint8_t *bits, float *post, uint8_t *conv, int32_t *it,
                     cudaStream_t st, bool out_dev) {
    return dispatch_w<float>(d, in, sigma, syn, batch, iters, et, bits, post, conv, it, st, out_dev);
}

}  // namespace mld
