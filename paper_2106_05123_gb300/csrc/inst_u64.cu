// Instantiation of the plain sort path for PDQ_U64 keys (keys only, 4-byte and 8-byte payloads).
#include "sort_impl.cuh"
PDQ_INSTANTIATE(PDQ_U64)
