// cv_sample_b.cu -- instantiates the sampling and Sobol kernels for
// ndim 9..16 (split over four files so they compile in parallel).
#include "cv_device.cuh"

CV_INSTANTIATE_NDIM(9)
CV_INSTANTIATE_NDIM(10)
CV_INSTANTIATE_NDIM(11)
CV_INSTANTIATE_NDIM(12)
CV_INSTANTIATE_NDIM(13)
CV_INSTANTIATE_NDIM(14)
CV_INSTANTIATE_NDIM(15)
CV_INSTANTIATE_NDIM(16)
