// cv_sample_6.cu -- instantiates the sampling, materialised-sample and Sobol
// kernels for ndim 7, 15, 23, 31 (the 32 dimension counts are spread over
// eight files, interleaved so the files take similar time, and compiled in
// parallel).
#include "cv_device.cuh"

CV_INSTANTIATE_NDIM(7)
CV_INSTANTIATE_NDIM(15)
CV_INSTANTIATE_NDIM(23)
CV_INSTANTIATE_NDIM(31)
