/* oracle_internal.h -- helpers shared by the oracle's own translation units (test infrastructure). */
#ifndef VR_ORACLE_INTERNAL_H
#define VR_ORACLE_INTERNAL_H
#include <stdint.h>

int or_threads(int threads);
void or_parallel_for(int64_t n, int64_t chunk, int threads, void (*fn)(void*, int64_t, int64_t), void* arg);

#endif
