// cv_sample_2.cu -- instantiates the sampling, materialised-sample and Sobol
// kernels for ndim 3, 11, 19, 27 (the 32 dimension counts are spread over
// eight files, interleaved so the files take similar time, and compiled in
// parallel).
#include "cv_device.cuh"

CV_INSTANTIATE_NDIM(3)
CV_INSTANTIATE_NDIM(11)
CV_INSTANTIATE_NDIM(19)
CV_INSTANTIATE_NDIM(27)
