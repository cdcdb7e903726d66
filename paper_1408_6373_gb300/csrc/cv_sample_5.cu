// cv_sample_5.cu -- instantiates the sampling, materialised-sample and Sobol
// kernels for ndim 6, 14, 22, 30 (the 32 dimension counts are spread over
// eight files, interleaved so the files take similar time, and compiled in
// parallel).
#include "cv_device.cuh"

CV_INSTANTIATE_NDIM(6)
CV_INSTANTIATE_NDIM(14)
CV_INSTANTIATE_NDIM(22)
CV_INSTANTIATE_NDIM(30)
