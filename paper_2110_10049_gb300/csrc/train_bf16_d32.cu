// Training-step kernel instantiations for bf16 storage, d = 32.
#include "train_kernels.cuh"

namespace gosh {
namespace {
using T = __nv_bfloat16;
constexpr int L0 = 32 * (int)sizeof(T) / 16;
constexpr gosh_dtype kType = GOSH_BF16;

#define GOSH_V(D, L, P, MODE) {kType, D, L, P, MODE, &make_train_kernel<T, D, L, P, MODE>}
#define GOSH_VD(D, L0)                                                                               \
    GOSH_V(D, L0, 2, kModeRed), GOSH_V(D, L0, 4, kModeRed), GOSH_V(D, L0 / 2, 2, kModeRed),          \
        GOSH_V(D, L0 / 2, 4, kModeRed), GOSH_V(D, L0, 2, kModeStore), GOSH_V(D, L0, 4, kModeStore),   \
        GOSH_V(D, L0 / 2, 2, kModeStore), GOSH_V(D, L0 / 2, 4, kModeStore), GOSH_V(D, L0, 4, kModeDet), \
        GOSH_V(D, L0, 8, kModeDet)

const TrainEntry kEntries[] = {GOSH_VD(32, L0)};
#undef GOSH_VD
#undef GOSH_V
}  // namespace

const TrainEntry *train_entries_bf16_d32(int *count) {
    *count = (int)(sizeof(kEntries) / sizeof(kEntries[0]));
    return kEntries;
}

}  // namespace gosh
