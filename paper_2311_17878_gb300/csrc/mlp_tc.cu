// BF16 tensor-core (tcgen05) evaluation of the networks: not built yet.
#include "common.cuh"

namespace tsdfs {
int mlp_tc_available(int arch) {
    (void)arch;
    return 0;
}
int launch_mlp_full_tc(const tsdfs_mlp*, const SampleSource&, SampleRec*, int64_t, cudaStream_t) {
    return fail(TSDFS_E_UNSUPPORTED, "BF16 tensor-core path not built");
}
}  // namespace tsdfs

using namespace tsdfs;

extern "C" size_t tsdfs_packed_size(int32_t arch) {
    (void)arch;
    return 0;
}
extern "C" int tsdfs_pack_mlp(const tsdfs_mlp* mlp, void* packed, tsdfs_stream_t stream) {
    (void)mlp;
    (void)packed;
    (void)stream;
    return fail(TSDFS_E_UNSUPPORTED, "BF16 tensor-core path not built");
}
