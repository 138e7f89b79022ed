// Training-step kernel instantiations for f16 storage, d = 8 (a 16-byte row:
// one lane per source, so a warp updates 32 sources at once).
#include "train_kernels.cuh"

namespace gosh {
namespace {
using T = __half;
constexpr gosh_dtype kType = GOSH_F16;

#define GOSH_V(D, L, P, MODE) {kType, D, L, P, MODE, &make_train_kernel<T, D, L, P, MODE>}
const TrainEntry kEntries[] = {GOSH_V(8, 1, 2, kModeRed),   GOSH_V(8, 1, 4, kModeRed), GOSH_V(8, 1, 2, kModeStore),
                               GOSH_V(8, 1, 4, kModeStore), GOSH_V(8, 1, 4, kModeDet), GOSH_V(8, 1, 8, kModeDet)};
#undef GOSH_V
}  // namespace

const TrainEntry *train_entries_f16_d8(int *count) {
    *count = (int)(sizeof(kEntries) / sizeof(kEntries[0]));
    return kEntries;
}

}  // namespace gosh
