// Instantiation of the plain and segmented sort paths for PDQ_I32I32 keys (composite 8-byte records;
// keys only, 4-byte and 8-byte payloads).
#include "seg_impl.cuh"
#include "sort_impl.cuh"
PDQ_INSTANTIATE(PDQ_I32I32)
PDQ_INSTANTIATE_SEG(PDQ_I32I32)
