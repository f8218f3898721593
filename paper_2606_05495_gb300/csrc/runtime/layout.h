// layout.h -- byte sizes and slot placement of every job type (host only, no CUDA headers).
#pragma once

#include <cstddef>
#include <cstdint>

namespace setk {

// A job occupies a slot as [control | in | out | scratch]:
//   control: persistent state a kernel keeps across launches (zeroed once when the slot is
//            created, never written by copies or by other job types, always at slot offset 0);
//   in/out : the H2D and D2H payloads; scratch: transient work buffers of this job.
// Each region starts on a 256-byte boundary.
struct JobLayout {
  size_t in_bytes = 0, out_bytes = 0, scratch_bytes = 0, persist_bytes = 0;
  size_t in_off = 0, out_off = 0, scratch_off = 0, end = 0;
};

inline size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// Sizes of one job; false if type or dims are invalid.
bool job_sizes(uint32_t type, const uint32_t dims[4], JobLayout* L);

// Control-block bytes reserved at the start of every slot of `slot_bytes`: enough for the
// persistent state of any job whose payload fits the slot.
size_t slot_control_bytes(size_t slot_bytes);

// Offset of a job type's persistent state inside the slot control block.
size_t control_offset(uint32_t type);

// Places the job's regions after a control block of `ctl` bytes.
void place_job(JobLayout* L, size_t ctl);

// Guarded placement (set_config.guards): a kGuardBytes band before `in` and one directly after
// each of in, out and scratch (at in_off + in_bytes etc.); regions still start 256-byte aligned.
constexpr size_t kGuardBytes = 256;
void place_job_guarded(JobLayout* L, size_t ctl);
// The four band offsets of a placed, guarded job.
void guard_offsets(const JobLayout& L, size_t off[4]);

// ---- batched form: several jobs of one type in one launch ----
constexpr int kMaxBatch = 64;

struct BatchItem {
  uint32_t dims[4];
  uint64_t job_id;
};

// One device block per batch: [table | job regions].  The table (job descriptors plus the
// zero-initialised transient state of the packed kernels) is written on the host and copied in
// by the batch graph's first node.
struct BatchLayout {
  int nb = 0;
  size_t table_bytes = 0, block_bytes = 0;
  size_t in_off[kMaxBatch], in_bytes[kMaxBatch], out_off[kMaxBatch], out_bytes[kMaxBatch];
  size_t rows = 0;  // MLP: packed rows (sum of m_j + 1)
};

// True for the job types that have a batched form (image, MLP).
bool batchable(uint32_t type);
bool batch_layout(uint32_t type, const BatchItem* items, int nb, BatchLayout* L);

}  // namespace setk
