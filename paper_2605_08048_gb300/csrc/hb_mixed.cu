// hb_mixed.cu -- tensor-core (tcgen05) group-sum path.  Placeholder until the
// kernel lands: the launcher reports that the path is not built.
#include <string>

#include "hb_internal.cuh"

namespace hb {
struct MixedArgs;
size_t mixed_work_bytes(int, const PairMeta *) { return 0; }
cudaError_t launch_mixed(const MixedArgs &, cudaStream_t, std::string &err)
{
    err = "the tensor-core path is not built in this version";
    return cudaErrorNotSupported;
}
}  // namespace hb
