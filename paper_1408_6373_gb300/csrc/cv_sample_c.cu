// cv_sample_c.cu -- instantiates the sampling and Sobol kernels for
// ndim 17..24 (split over four files so they compile in parallel).
#include "cv_device.cuh"

CV_INSTANTIATE_NDIM(17)
CV_INSTANTIATE_NDIM(18)
CV_INSTANTIATE_NDIM(19)
CV_INSTANTIATE_NDIM(20)
CV_INSTANTIATE_NDIM(21)
CV_INSTANTIATE_NDIM(22)
CV_INSTANTIATE_NDIM(23)
CV_INSTANTIATE_NDIM(24)
