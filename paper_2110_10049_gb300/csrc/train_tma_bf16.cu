// TMA-staged lock-free training kernels for bf16 tables.
#include "train_tma.cuh"

namespace gosh {
namespace {
using T = __nv_bfloat16;
constexpr gosh_dtype kType = GOSH_BF16;

#define GOSH_TV(D, L, KS) {kType, D, L, -(KS), kModeRed, &make_train_tma_kernel<T, D, L, KS, kModeRed>}
#define GOSH_TVL(D, L) GOSH_TV(D, L, 4), GOSH_TV(D, L, 6)
#define GOSH_TVD(D, L0a, L0b) GOSH_TVL(D, L0a), GOSH_TVL(D, L0b)
constexpr int L032 = 32 * (int)sizeof(T) / 16, L064 = 64 * (int)sizeof(T) / 16, L0128 = 128 * (int)sizeof(T) / 16;
const TrainEntry kEntries[] = {GOSH_TVD(32, L032, L032 / 2), GOSH_TVD(64, L064 / 2, L064 / 4),
                               GOSH_TVD(128, L0128 / 2, L0128 / 4)};
#undef GOSH_TVD
#undef GOSH_TVL
#undef GOSH_TV
}  // namespace

const TrainEntry *train_tma_entries_bf16(int *count) {
    *count = (int)(sizeof(kEntries) / sizeof(kEntries[0]));
    return kEntries;
}

}  // namespace gosh
