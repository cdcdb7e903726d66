// cv_sample_0.cu -- instantiates the sampling, materialised-sample and Sobol
// kernels for ndim 1, 9, 17, 25 (the 32 dimension counts are spread over
// eight files, interleaved so the files take similar time, and compiled in
// parallel).
#include "cv_device.cuh"

CV_INSTANTIATE_NDIM(1)
CV_INSTANTIATE_NDIM(9)
CV_INSTANTIATE_NDIM(17)
CV_INSTANTIATE_NDIM(25)
