// cv_sample_6.cu -- instantiates the sampling, materialised-sample and Sobol
// kernels for ndim 7 and 23 (the 32 dimension counts are spread over
// sixteen files, a small count with a large one so the files take similar
// time, and compiled in parallel).
#include "cv_device.cuh"

CV_INSTANTIATE_NDIM(7)
CV_INSTANTIATE_NDIM(23)
