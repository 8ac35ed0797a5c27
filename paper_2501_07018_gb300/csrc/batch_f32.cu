// FP32-bulk instantiation of the persistent batch kernel (batch_impl.cuh); its own
// translation unit so that the two precisions compile in parallel.
#include "batch_impl.cuh"

namespace pdlp {

int batch_config_count() { return kNumConfigs; }

template int batch_resident_ctas<float>(int);
template void launch_batch<float>(const BatchLP<float>*, const int32_t*, int, const BatchParams&,
                                  BatchResult*, unsigned int*, int, int, cudaStream_t);

}  // namespace pdlp
