// capi.cpp -- the extern "C" executor entry points declared in include/set.h.
#include <cstring>
#include <string>

#include "executor.h"
#include "layout.h"
#include "set.h"
#include "thread_error.h"

struct set_ctx {
  setrt::Executor* ex;
};

namespace {
thread_local std::string g_err;

set_status ctx_less(set_status st, const std::string& msg) {
  g_err = msg;
  return st;
}
}  // namespace

namespace setrt {
void set_thread_error(const char* msg) { g_err = msg ? msg : ""; }
const char* thread_error_text() { return g_err.c_str(); }
}  // namespace setrt

extern "C" {

size_t set_job_in_bytes(uint32_t type, const uint32_t dims[4]) {
  setk::JobLayout L;
  return dims && setk::job_sizes(type, dims, &L) ? L.in_bytes : 0;
}

size_t set_job_out_bytes(uint32_t type, const uint32_t dims[4]) {
  setk::JobLayout L;
  return dims && setk::job_sizes(type, dims, &L) ? L.out_bytes : 0;
}

size_t set_job_scratch_bytes(uint32_t type, const uint32_t dims[4]) {
  setk::JobLayout L;
  if (!dims || !setk::job_sizes(type, dims, &L)) return 0;
  return setk::align256(L.persist_bytes) + L.scratch_bytes;
}

size_t set_job_slot_bytes(uint32_t type, const uint32_t dims[4]) {
  setk::JobLayout L;
  if (!dims || !setk::job_sizes(type, dims, &L)) return 0;
  size_t s = 4096;
  for (int it = 0; it < 8; ++it) {  // the control block grows (slowly) with the slot
    setk::JobLayout P = L;
    setk::place_job(&P, setk::slot_control_bytes(s));
    if (P.end <= s) break;
    s = P.end;
  }
  return s;
}

void set_config_default(set_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof *c);
  c->num_streams = 2;
  c->num_workers = 2;
  c->slot_bytes = 1u << 20;
  c->ring_depth = 2;
  c->queue_capacity = 4;
  c->steal = 1;
  c->io_mode = SET_IO_HOST;
  c->img_fused = 1;
  c->type_mask = 0;
  c->device = 0;
  c->drain_timeout_ms = 30000;
  c->cb_mode = 0;
  c->spin_us = 50;
  c->cb_every = 1;
  c->batch_max = 1;
  c->img_ctas_per_sm = 4;
  c->img_tile = 0;
  c->stamps = 0;
  c->arena_bytes = 0;
}

set_status set_create_ex(const set_config* cfg, set_ctx** out) {
  if (!cfg || !out) return ctx_less(SET_EINVAL, "null argument");
  setrt::Executor* ex = nullptr;
  std::string err;
  const set_status st = setrt::Executor::create(*cfg, &ex, &err);
  if (st != SET_OK) return ctx_less(st, err);
  *out = new set_ctx{ex};
  return SET_OK;
}

set_status set_create(int num_streams, int num_workers, size_t slot_bytes, set_ctx** out) {
  set_config c;
  set_config_default(&c);
  c.num_streams = num_streams;
  c.num_workers = num_workers;
  c.slot_bytes = slot_bytes;
  return set_create_ex(&c, out);
}

set_status set_submit(set_ctx* ctx, const set_job_desc* job, uint64_t* job_id) {
  if (!ctx || !job) return ctx_less(SET_EINVAL, "null argument");
  return ctx->ex->submit(job, job_id);
}

set_status set_submit_many(set_ctx* ctx, const set_job_desc* jobs, size_t n, uint64_t* first_id, size_t* n_done) {
  if (!ctx || (!jobs && n)) return ctx_less(SET_EINVAL, "null argument");
  return ctx->ex->submit_many(jobs, n, first_id, n_done);
}

set_status set_wait_all(set_ctx* ctx, int64_t timeout_us) {
  if (!ctx) return ctx_less(SET_EINVAL, "null argument");
  return ctx->ex->wait_all(timeout_us);
}

set_status set_stats(set_ctx* ctx, set_stats_t* out) {
  if (!ctx || !out) return ctx_less(SET_EINVAL, "null argument");
  ctx->ex->stats(out);
  return SET_OK;
}

set_status set_reset_stats(set_ctx* ctx) {
  if (!ctx) return ctx_less(SET_EINVAL, "null argument");
  ctx->ex->reset_stats();
  return SET_OK;
}

set_status set_destroy(set_ctx* ctx) {
  if (!ctx) return ctx_less(SET_EINVAL, "null argument");
  delete ctx->ex;
  delete ctx;
  return SET_OK;
}

const char* set_last_error(set_ctx* ctx) {
  if (!ctx) return g_err.c_str();
  return ctx->ex->last_error();
}

set_status set_autotune(set_ctx* ctx, uint32_t type, const set_job_desc* sample, size_t n, set_tune_result* out) {
  if (!ctx) return ctx_less(SET_EINVAL, "null argument");
  return ctx->ex->autotune(type, sample, n, out);
}

set_status set_serve(set_ctx* ctx, int mode, const set_job_desc* jobs, const uint64_t* arrival_ns, size_t n,
                     set_stats_t* out) {
  if (!ctx) return ctx_less(SET_EINVAL, "null argument");
  return ctx->ex->serve(mode, jobs, arrival_ns, n, out);
}

set_status set_run_baseline(set_ctx* ctx, int kind, const set_job_desc* jobs, size_t n, set_stats_t* out) {
  if (!ctx) return ctx_less(SET_EINVAL, "null argument");
  return ctx->ex->run_baseline(kind, jobs, n, out);
}

}  // extern "C"
