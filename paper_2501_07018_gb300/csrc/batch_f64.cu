// FP64 instantiation of the persistent batch kernel (batch_impl.cuh); its own
// translation unit so that the two precisions compile in parallel.
#include "batch_impl.cuh"

namespace pdlp {

template int batch_resident_ctas<double>(int);
template void launch_batch<double>(const BatchLP<double>*, const int32_t*, int, const BatchParams&,
                                   BatchResult*, unsigned int*, int, int, cudaStream_t);

}  // namespace pdlp
