// cv_sample_d.cu -- instantiates the sampling and Sobol kernels for
// ndim 25..32 (split over four files so they compile in parallel).
#include "cv_device.cuh"

CV_INSTANTIATE_NDIM(25)
CV_INSTANTIATE_NDIM(26)
CV_INSTANTIATE_NDIM(27)
CV_INSTANTIATE_NDIM(28)
CV_INSTANTIATE_NDIM(29)
CV_INSTANTIATE_NDIM(30)
CV_INSTANTIATE_NDIM(31)
CV_INSTANTIATE_NDIM(32)
