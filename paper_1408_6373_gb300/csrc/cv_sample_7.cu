// cv_sample_7.cu -- instantiates the sampling, materialised-sample and Sobol
// kernels for ndim 8, 16, 24, 32 (the 32 dimension counts are spread over
// eight files, interleaved so the files take similar time, and compiled in
// parallel).
#include "cv_device.cuh"

CV_INSTANTIATE_NDIM(8)
CV_INSTANTIATE_NDIM(16)
CV_INSTANTIATE_NDIM(24)
CV_INSTANTIATE_NDIM(32)
