// cv_sample_1.cu -- instantiates the sampling, materialised-sample and Sobol
// kernels for ndim 2, 10, 18, 26 (the 32 dimension counts are spread over
// eight files, interleaved so the files take similar time, and compiled in
// parallel).
#include "cv_device.cuh"

CV_INSTANTIATE_NDIM(2)
CV_INSTANTIATE_NDIM(10)
CV_INSTANTIATE_NDIM(18)
CV_INSTANTIATE_NDIM(26)
