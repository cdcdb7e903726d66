// cv_sample_4.cu -- instantiates the sampling, materialised-sample and Sobol
// kernels for ndim 5, 13, 21, 29 (the 32 dimension counts are spread over
// eight files, interleaved so the files take similar time, and compiled in
// parallel).
#include "cv_device.cuh"

CV_INSTANTIATE_NDIM(5)
CV_INSTANTIATE_NDIM(13)
CV_INSTANTIATE_NDIM(21)
CV_INSTANTIATE_NDIM(29)
