// float64 instantiation of the spreading / interpolation kernels.
using real_t = double;
#include "dispatch_impl.cuh"
