// The double-float FFT kernels of the FP64 plans at P = 4096 (band limit 1024); see df_fft.cuh.
#include "df_fft_impl.cuh"

CRV_DF_DEFINE(4096)
