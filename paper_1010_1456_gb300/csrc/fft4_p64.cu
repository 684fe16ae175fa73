// Four-step FFT kernels for the P64 policy (see fft4.cuh).
#include "common.h"
#define AIM_FFT4_POLICY P64
#define AIM_FFT4_NAME(k) fft4_##k##_p64
#include "fft4_launch.cuh"
