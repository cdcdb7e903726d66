// cv_sample_3.cu -- instantiates the sampling, materialised-sample and Sobol
// kernels for ndim 4, 12, 20, 28 (the 32 dimension counts are spread over
// eight files, interleaved so the files take similar time, and compiled in
// parallel).
#include "cv_device.cuh"

CV_INSTANTIATE_NDIM(4)
CV_INSTANTIATE_NDIM(12)
CV_INSTANTIATE_NDIM(20)
CV_INSTANTIATE_NDIM(28)
