// The batched persistent kernel at 128 threads per CTA (mhd_batch.cuh).
#include "mhd_batch.cuh"

MHD_BATCH_INSTANTIATE(128)
