// Training-step kernel instantiations for f32 storage.
#include "train_kernels.cuh"

namespace gosh {
namespace {
using T = float;
constexpr int L8 = 8 * (int)sizeof(T) / 16;
constexpr int L16 = 16 * (int)sizeof(T) / 16;
constexpr int L32 = 32 * (int)sizeof(T) / 16;
constexpr int L64 = 64 * (int)sizeof(T) / 16;
constexpr int L128 = 128 * (int)sizeof(T) / 16;
constexpr gosh_dtype kType = GOSH_F32;

#define GOSH_V(D, L, P, MODE) {kType, D, L, P, MODE, &make_train_kernel<T, D, L, P, MODE>}
#define GOSH_VD(D, L0)                                                                               \
    GOSH_V(D, L0, 2, kModeRed), GOSH_V(D, L0, 4, kModeRed), GOSH_V(D, L0 / 2, 2, kModeRed),          \
        GOSH_V(D, L0 / 2, 4, kModeRed), GOSH_V(D, L0, 4, kModeStore), GOSH_V(D, L0, 4, kModeDet),     \
        GOSH_V(D, L0, 8, kModeDet)

const TrainEntry kEntries[] = {GOSH_VD(8, L8), GOSH_VD(16, L16), GOSH_VD(32, L32), GOSH_VD(64, L64),
                               GOSH_VD(128, L128)};
#undef GOSH_VD
#undef GOSH_V
}  // namespace

const TrainEntry *train_entries_f32(int *count) {
    *count = (int)(sizeof(kEntries) / sizeof(kEntries[0]));
    return kEntries;
}

void det_apply_f32(int d, const uint32_t *skeys, const uint32_t *sidx, int64_t nslots, const float *C,
                  const float *R, void *M, int64_t n, int64_t b0, int64_t b1, uint8_t *src_done,
                  uint32_t sr_seed, cudaStream_t s) {
    switch (d) {
    case 8: launch_det_apply_t<T, 8>(skeys, sidx, nslots, C, R, M, n, b0, b1, src_done, sr_seed, s); break;
    case 16: launch_det_apply_t<T, 16>(skeys, sidx, nslots, C, R, M, n, b0, b1, src_done, sr_seed, s); break;
    case 32: launch_det_apply_t<T, 32>(skeys, sidx, nslots, C, R, M, n, b0, b1, src_done, sr_seed, s); break;
    case 64: launch_det_apply_t<T, 64>(skeys, sidx, nslots, C, R, M, n, b0, b1, src_done, sr_seed, s); break;
    case 128: launch_det_apply_t<T, 128>(skeys, sidx, nslots, C, R, M, n, b0, b1, src_done, sr_seed, s); break;
    default: break;
    }
}

}  // namespace gosh
