// pinned.cuh -- the library's page-locked host blocks.
//
// Allocating page-locked host memory is an implicit synchronisation point of the device:
// commands of different streams cannot overlap across it.  A serving process whose worker
// threads set up, solve and free hierarchies on their own streams would serialise all of
// them at every setup, so the small readback buffers of handles and batches come from one
// process-wide free list instead: power-of-two blocks, allocated once, reused, and never
// returned to the driver.  A block goes back to the list only once no copy into it is in
// flight (the caller synchronises its stream first).
#pragma once
#include <cstddef>

namespace uaamg {

// A page-locked block of at least `bytes` bytes, or nullptr when the driver has none.
void* pinned_get(size_t bytes);
// Returns a block from pinned_get to the free list (nullptr is ignored).
void pinned_put(void* p);

}  // namespace uaamg
