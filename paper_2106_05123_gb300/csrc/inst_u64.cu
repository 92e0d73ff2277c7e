// Instantiation of the plain sort path for PDQ_U64 keys (keys only, 4-byte and 8-byte payloads; plain and segmented).
#include "seg_impl.cuh"
#include "sort_impl.cuh"
PDQ_INSTANTIATE(PDQ_U64)
PDQ_INSTANTIATE_SEG(PDQ_U64)
