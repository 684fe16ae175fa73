// Four-step FFT kernels for the PFF policy (see fft4.cuh).
#include "common.h"
#define AIM_FFT4_POLICY PFF
#define AIM_FFT4_NAME(k) fft4_##k##_pff
#include "fft4_launch.cuh"
