// cv_sample_a.cu -- instantiates the sampling and Sobol kernels for
// ndim 1..8 (split over four files so they compile in parallel).
#include "cv_device.cuh"

CV_INSTANTIATE_NDIM(1)
CV_INSTANTIATE_NDIM(2)
CV_INSTANTIATE_NDIM(3)
CV_INSTANTIATE_NDIM(4)
CV_INSTANTIATE_NDIM(5)
CV_INSTANTIATE_NDIM(6)
CV_INSTANTIATE_NDIM(7)
CV_INSTANTIATE_NDIM(8)
