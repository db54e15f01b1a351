// Host-side helpers shared by the C-ABI translation units (internal; not part of the C ABI).
#pragma once
#include <cstdint>

#include "turtle.h"

// Host-memory form of turtle_count on a given context (copies or streams the reads in).
int count_host_impl(turtle_ctx *c, const turtle_reads *reads, int k, uint32_t min_count, const turtle_params *params,
                    void *stream, turtle_result *out);

// Upper estimate of the device memory one call needs for n_bases bases (no key-range split):
// the reads, their packed form and bitmaps, and the per-window buffers of the post-filter stages.
uint64_t footprint_estimate(uint64_t n_bases, uint64_t n_reads, int k, uint32_t min_count, const turtle_params *p);
