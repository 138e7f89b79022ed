// Training-step kernel instantiations for bf16 storage: one translation
// unit per embedding width (train_bf16_d<d>.cu, compiled in parallel), and
// here the list of all of them and the deterministic-mode apply kernels.
#include <vector>

#include "train_kernels.cuh"

namespace gosh {

const TrainEntry *train_entries_bf16_d8(int *count);
const TrainEntry *train_entries_bf16_d16(int *count);
const TrainEntry *train_entries_bf16_d32(int *count);
const TrainEntry *train_entries_bf16_d64(int *count);
const TrainEntry *train_entries_bf16_d128(int *count);

const TrainEntry *train_entries_bf16(int *count) {
    static std::vector<TrainEntry> all = [] {
        std::vector<TrainEntry> v;
        for (auto f : {train_entries_bf16_d8, train_entries_bf16_d16, train_entries_bf16_d32, train_entries_bf16_d64,
                       train_entries_bf16_d128}) {
            int c = 0;
            const TrainEntry *e = f(&c);
            v.insert(v.end(), e, e + c);
        }
        return v;
    }();
    *count = (int)all.size();
    return all.data();
}

namespace {
using T = __nv_bfloat16;
}  // namespace

void det_apply_bf16(int d, const uint32_t *skeys, const uint32_t *sidx, int64_t nslots, const float *C,
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
