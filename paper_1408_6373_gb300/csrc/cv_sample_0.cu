// cv_sample_0.cu -- instantiates the sampling, materialised-sample and Sobol
// kernels for ndim 1 and 17 (the 32 dimension counts are spread over
// sixteen files, a small count with a large one so the files take similar
// time, and compiled in parallel).
#include "cv_device.cuh"

CV_INSTANTIATE_NDIM(1)
CV_INSTANTIATE_NDIM(17)
