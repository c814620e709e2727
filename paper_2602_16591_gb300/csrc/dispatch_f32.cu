// float32 instantiation of the spreading / interpolation kernels.
using real_t = float;
#include "dispatch_impl.cuh"
