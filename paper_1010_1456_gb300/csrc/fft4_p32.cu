// Four-step FFT kernels for the P32 policy (see fft4.cuh).
#include "common.h"
#define AIM_FFT4_POLICY P32
#define AIM_FFT4_NAME(k) fft4_##k##_p32
#include "fft4_launch.cuh"
