// The double-float FFT kernels of the FP64 plans at P = 2048 (band limit 512); see df_fft.cuh.
#include "df_fft_impl.cuh"

CRV_DF_DEFINE(2048)
