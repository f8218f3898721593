// dev_dispatch.h -- memory layout shared by the host side of the device-dispatch lanes and their
// fetch kernel.
//
// A lane is one stream running one graph: WHILE { fetch -> SWITCH(kind) { blur | scan | image } }.
// The host writes job descriptors into the lane's ring (page-locked host memory the GPU reads
// over the host link); the fetch kernel of each iteration retires the job the previous iteration
// ran (completion words and counter into host memory), waits a bounded time for the next
// descriptor, copies its kernel arguments (and those of the same-kind descriptors queued behind
// it, up to kDdBatch) into the lane's device block and selects the kind for the SWITCH node.  No descriptor within the idle limit: it ends the loop and counts an exit.
#pragma once

#include <cstddef>
#include <cstdint>

#include "set.h"

namespace setk {

constexpr uint32_t kDdKindBlur = 0, kDdKindScan = 1, kDdKindImg = 2, kDdKinds = 3;
constexpr uint32_t kDdKindNone = 7;  // >= the SWITCH node's body count: no body runs
constexpr size_t kDdArgBytes = 192;
// Jobs one loop iteration may take at once: consecutive blur or scan descriptors of the same kind
// already waiting in the ring run as one launch of their node (job j of the batch on the j-th
// group of the node's grid: a cluster of the blur node, a tile range of the scan node with its
// own look-back scratch).  Image jobs run one per iteration (their node's grid pulls the tiles of
// one image from the lane's ticket).
constexpr uint32_t kDdBatch = 8;

// One ring entry: 32 8-byte words, read by the fetch kernel's warp with one word per thread.
// The host fills words 1..31, then stores seq (word 0) with release order.
struct alignas(64) DdEntry {
  uint64_t seq;           // position in the lane's sequence + 1 once the entry is complete
  uint32_t kind;          // kDdKind*
  uint32_t args_size;     // bytes of args used
  uint64_t job_id;        // echoed in the trailer the job's kernel writes
  set_trailer* trailer;   // the job's trailer (device-usable address)
  uint64_t pad[4];
  unsigned char args[kDdArgBytes];  // the stage kernel's argument struct
};
static_assert(sizeof(DdEntry) == 256, "one entry = 32 words of 8 bytes");

// Per-lane control words in host memory (one 64-byte line each).
struct alignas(64) DdCtl {
  uint64_t done;   // device -> host: jobs of this lane retired (release order)
  uint32_t exits;  // device -> host: times the lane's loop has ended
  uint32_t stop;   // host -> device: end the loop at the next fetch
  uint64_t pad[6];
};
static_assert(sizeof(DdCtl) == 64, "one line per lane");

// Per-lane state in device memory, kept across launches of the lane's graph.
struct alignas(64) DdLaneDev {
  uint64_t head;       // descriptors fetched so far
  uint64_t cur_first;  // sequence + 1 of the first job in flight (0: none to retire)
  uint32_t cur_count;  // jobs in flight (consecutive sequences)
  uint32_t exits;      // loop exits so far (mirrors DdCtl::exits)
  uint32_t batch_count; // jobs in batch_args this iteration (read by the blur or scan kernel)
  uint32_t pad0;
  uint64_t pad1[4];
  uint64_t cur_job[kDdBatch];          // job ids in flight
  set_trailer* cur_trailer[kDdBatch];  // their trailers
  alignas(64) unsigned char args[kDdKinds][kDdArgBytes];        // a kind that runs one job (image)
  alignas(64) unsigned char batch_args[kDdBatch][kDdArgBytes];  // the blur or scan jobs of the batch
};

struct DdFetchArgs {
  DdLaneDev* lane;
  const DdEntry* ring;  // device-usable address of the lane's ring
  DdCtl* ctl;           // device-usable address of the lane's control line
  uint32_t* cmpl;       // device-usable address of the lane's completion words (one per ring entry)
  uint32_t depth;       // ring entries (power of two)
  uint32_t pad;
  uint64_t idle_ns;     // end the loop after this long without a descriptor
  unsigned long long loop;  // cudaGraphConditionalHandle of the WHILE node's condition
  unsigned long long kind;  // cudaGraphConditionalHandle of the SWITCH node's selector
};

}  // namespace setk
