/*
 * set.h -- C ABI of the stream-event-triggered (SET) job executor for one GB300 (sm_103a).
 *
 * The executor follows Sec. 4 of "SET: Stream-Event-Triggered Scheduling for Efficient CUDA
 * Graph Pipelines" (Li, Huang, Ogras):
 *   - a job is a reusable CUDA graph: H2D copy -> chain or DAG of stage kernels -> D2H copy,
 *     with per-job arguments held as placeholders and updated at run time (Sec. 4.1);
 *   - each lane (the paper's worker W_i, Sec. 4.2 "Scheduler Components") owns a stream and a
 *     ring of slots; a slot is a pre-allocated device buffer M with one pre-instantiated graph
 *     executable G per job type bound to it, so G touches only M (Sec. 4.1, 4.2);
 *   - per-lane bounded job queues Q_i and a lock-free free-slot pool W_pool (Sec. 4.2);
 *   - set_submit is the job submitter (Algorithm 1);
 *   - host dispatch workers pop a free slot, take a job from the slot's lane queue or steal one
 *     from lane (w+k) mod b, retarget it to the slot (UpdateGraphParams through
 *     cudaGraphExecKernelNodeSetParams / cudaGraphExecMemcpyNodeSetParams1D), launch the graph
 *     and chain a completion callback to it (Algorithm 2);
 *   - the completion callback, run by the CUDA driver through cudaLaunchHostFunc after an event
 *     recorded behind the graph, counts the job done and returns the slot to W_pool
 *     (Algorithm 3).  The lane stream itself never waits on the host.  set_config.cb_mode 3
 *     runs the same completion code on a thread of the context that polls each lane's oldest
 *     event instead (an addition: lower latency than the driver's callback thread).
 *
 * Conventions (every function):
 *   - The return value is the status; nothing throws across this boundary.
 *   - A CUDA error inside a context is sticky: later calls on that context return SET_ECUDA and
 *     set_last_error() gives the CUDA error text.
 *   - Host input / output buffers belong to the caller and must stay valid until the job
 *     completes.  With SET_IO_HOST and the mapped modes they must be page-locked (cudaHostAlloc
 *     or a pinned torch tensor); with SET_IO_DEVICE and SET_IO_DEVICE_INPLACE they must be device
 *     pointers of the context's GPU.
 *   - Device memory of the slot pool belongs to the context, or to the caller when passed in
 *     set_config.pool / pool_bytes (for example a torch tensor).
 *   - Thread safety: set_submit, set_submit_many, set_wait_all and set_stats may be called from
 *     any number of threads.  set_destroy must not race with any other call on the context.
 */
#ifndef SET_H_
#define SET_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct set_ctx set_ctx; /* opaque: streams, graph execs, slots, queues, threads */

typedef enum {
  SET_OK = 0,
  SET_EINVAL = -1,     /* bad argument or descriptor (type, sizes, null pointer, pageable host memory) */
  SET_ENOMEM = -2,     /* job does not fit a slot, or the slot pool cannot be allocated */
  SET_EAGAIN = -3,     /* every lane queue is full and SET_F_NONBLOCK was given */
  SET_ETIMEDOUT = -4,  /* a bounded wait ran out */
  SET_ECUDA = -5,      /* CUDA runtime error; sticky for the context, text in set_last_error */
  SET_ESHUTDOWN = -6,  /* the context is being destroyed */
  SET_EDEVICE = -7     /* a device-side check failed for that job: a bounded wait gave up or the
                          returned trailer did not carry the job's id and slot generation */
} set_status;

/* Job types and their payload layouts.  "in" and "out" are the bytes of the H2D and D2H copies.
 * Every out ends with a 16-byte set_trailer written by the job's last kernel.
 *
 * SET_JOB_BLUR_HIST       dims = {W, H}, 1 <= W <= 2048, 1 <= H <= 65535.
 *   in : uint8 image, H rows of W bytes.
 *   out: blurred uint8 image (W*H bytes, o = floor(sum of the 9 edge-clamped neighbours / 9)),
 *        zero pad to 16 bytes, uint32 hist[256] of the blurred image, trailer.
 * SET_JOB_SAXPY_SCAN_MAX  dims = {n}, 1 <= n <= 2^26; scalar = a.
 *   in : float x[n] followed by float y[n].
 *   out: float z[n] (z_i = fmaf(a, x_i, y_i)), float S[n] (exclusive prefix sum of z, fp32),
 *        float m (max_i |S_i|), 12 zero bytes, trailer.
 * SET_JOB_IMG_SOBEL_HIST  dims = {W, H}, 1 <= W, H <= 4096.
 *   in : interleaved RGB uint8, H rows of 3*W bytes.
 *   out: Sobel uint8 image (W*H bytes) of gray -> 5x5 Gaussian -> Sobel, each stage clamping
 *        its own input at the border, zero pad to 16 bytes, uint32 hist[256], trailer.
 * SET_JOB_MLP_LN          dims = {m}, 1 <= m <= 256; shared[0] = W1, shared[1] = W2 (device).
 *   in : bf16 x[m][1024].
 *   out: float out[m][1024] = GELU(x W1^T) W2^T + LayerNorm(x), then the trailer.
 *        W1 is bf16 [4096][1024], W2 bf16 [1024][4096] (out_features x in_features), both
 *        device-resident and owned by the caller.  The job is a fork/join DAG.
 * SET_JOB_HOTSPOT         dims = {C, R, K}, 1 <= C, R <= 8192, 1 <= K <= 64.
 *   in : float T0[R][C] (temperatures) followed by float P[R][C] (watts per cell).
 *   out: float T[R][C] after K explicit steps of the compact thermal RC grid (die 16 mm x 16 mm
 *        x 0.5 mm, k = 100 W/(m K), c_v = 1.75e6 J/(m^3 K), T_amb = 80, step a fifth of the
 *        positivity limit, adiabatic edges), zero pad to 16 bytes, trailer.  A chain of 8
 *        kernels (K/8 steps each, rounded).
 */
typedef enum {
  SET_JOB_BLUR_HIST = 1,
  SET_JOB_SAXPY_SCAN_MAX = 2,
  SET_JOB_IMG_SOBEL_HIST = 3,
  SET_JOB_MLP_LN = 4,
  SET_JOB_HOTSPOT = 5
} set_job_type;

#define SET_NUM_JOB_TYPES 5

/* set_job_desc.flags */
#define SET_F_NONBLOCK 0x1u /* set_submit returns SET_EAGAIN instead of waiting for queue room */
#define SET_F_PER_STAGE 0x2u /* set_launch_job: run an image job as its three-stage chain (gray,
                                Gaussian, Sobel + histogram) instead of the fused kernel; contexts
                                choose with set_config.img_fused */
#define SET_F_TEST_GUARD 0x200u /* test hook for set_config.guards: the guard-arming kernel writes one
                                   wrong byte into the band after `out`, so the check must report
                                   SET_DEVERR_GUARD for this job (no kernel touches the band) */
#define SET_F_TEST_STALL 0x100u /* test hook for failure detection without a GPU fault: in a scan
                                   job of >= 3 tiles, tile 1 exits without publishing, so tile 2's
                                   look-back and the final max gather wait until their bounded
                                   limit (~0.1-0.4 s) runs out; the job completes with SET_EDEVICE
                                   (trailer error bit SET_DEVERR_WAIT) and the context stays usable */

/* The last 16 bytes of every job's output. */
typedef struct {
  uint64_t job_id;   /* id set_submit returned for this job */
  uint32_t slot_gen; /* generation of the slot that ran it (bumped at each completion) */
  uint32_t word;     /* (SET_TRAILER_MAGIC << 16) | device error bits */
} set_trailer;

#define SET_TRAILER_MAGIC 0x5E7Cu
#define SET_DEVERR_WAIT 0x1u /* a bounded device-side wait gave up */
#define SET_DEVERR_GUARD 0x2u /* set_config.guards: a guard band next to the job's regions changed */

typedef struct {
  uint32_t type;          /* set_job_type */
  uint32_t flags;         /* SET_F_* */
  const void* in;         /* caller-owned input (pinned host, or device with SET_IO_DEVICE) */
  size_t in_bytes;        /* must equal set_job_in_bytes(type, dims) */
  void* out;              /* caller-owned output, written only by the D2H copy */
  size_t out_bytes;       /* must equal set_job_out_bytes(type, dims) */
  uint32_t dims[4];       /* per type, see above; unused entries 0 */
  float scalar;           /* SET_JOB_SAXPY_SCAN_MAX: a */
  uint32_t reserved;      /* 0 */
  const void* shared[2];  /* SET_JOB_MLP_LN: device W1, W2; otherwise NULL */
  uint64_t user_tag;      /* opaque, kept with the job */
  uint64_t t_arrival_ns;  /* arrival time (CLOCK_MONOTONIC ns) latency is measured from; 0 = at submit */
  volatile int32_t* status; /* optional: set to a set_status when the job completes */
} set_job_desc;

/* Input / output placement of every job of a context.
 *   SET_IO_HOST    in / out are page-locked host buffers, moved by the graph's H2D / D2H copy
 *                  nodes (the paper's job: H2D -> kernels -> D2H).
 *   SET_IO_DEVICE  in / out are device buffers of the context's GPU (device-to-device copies).
 *   SET_IO_MAPPED  in / out are page-locked host buffers mapped into the GPU's address space
 *                  (cudaHostAlloc, a pinned torch tensor); the stage kernels read and write them
 *                  directly over the host link, so a job's graph has no copy nodes.  An addition
 *                  for hosts coherently attached to the GPU (NVLink-C2C); not for MLP jobs,
 *                  whose x feeds TMA loads (SET_EINVAL), nor for the batched form or baselines.
 *                  Buffers the device cannot address, and device memory (the completion path
 *                  reads the trailer on the host), are rejected at submit with SET_EINVAL.
 *   SET_IO_MAPPED_IN   in as SET_IO_MAPPED (no H2D node), out by the D2H copy node.
 *   SET_IO_MAPPED_OUT  in by the H2D copy node, out as SET_IO_MAPPED (the kernels store the job's
 *                  results straight into the pinned host buffer; no D2H node).  MLP jobs allowed.
 *   SET_IO_DEVICE_INPLACE  in / out are 16-byte aligned device buffers of the context's GPU that the
 *                  stage kernels read and write in place: the graph is the kernel DAG alone, no
 *                  copy nodes (the HBM-resident counterpart of SET_IO_MAPPED).  Not for MLP
 *                  jobs, the batched form or baselines (SET_EINVAL).  The trailer stays in the
 *                  caller's device buffer, as with SET_IO_DEVICE. */
typedef enum {
  SET_IO_HOST = 0,
  SET_IO_DEVICE = 1,
  SET_IO_MAPPED = 2,
  SET_IO_MAPPED_IN = 3,
  SET_IO_MAPPED_OUT = 4,
  SET_IO_DEVICE_INPLACE = 5
} set_io_mode;

typedef struct {
  int num_streams;     /* lanes b (paper's workers), >= 1 */
  int num_workers;     /* host dispatch threads, >= 1 */
  size_t slot_bytes;   /* bytes per slot: must cover in + out + scratch of the largest job */
  int ring_depth;      /* slots per lane (default 2): jobs a lane may hold in flight */
  int queue_capacity;  /* per-lane job queue capacity (default 4, rounded up to a power of 2) */
  int steal;           /* 1 (default): FindJob steals from other lanes; 0: local queue only */
  int io_mode;         /* set_io_mode of every job */
  int img_fused;       /* 1 (default): image jobs run one fused stencil kernel; 0: per stage */
  void* pool;          /* optional caller-owned device memory for the slots (else cudaMalloc) */
  size_t pool_bytes;   /* its size: >= num_streams * ring_depth * slot_bytes */
  uint32_t type_mask;  /* bit (1 << type) per job type to instantiate graphs for; 0 = all */
  int device;          /* CUDA device ordinal (default 0) */
  int drain_timeout_ms; /* set_destroy waits at most this long for jobs in flight (default 30000) */
  int cb_mode;         /* 0 (default): completion callback on a per-lane callback stream that waits
                          on an event recorded behind the graph (the lane never waits on the host);
                          1: cudaLaunchHostFunc directly on the lane stream;
                          2: a host node at the end of every slot's graph (no extra call per job);
                          3: no host function: an event recorded behind the graph, polled by a
                          completion thread of the context that runs the completion path (lower
                          latency, one host core busy while jobs are in flight) */
  int spin_us;         /* dispatch workers spin this long on an empty pool / queue before they
                          sleep on a futex (default 50; 0 = sleep at once) */
  int cb_every;        /* cb_mode 0/1/3: attach one completion callback per this many jobs of a lane
                          (it completes the whole group in stream order; default 1 = one per job).
                          Groups are closed early whenever a dispatch worker would wait. */
  int batch_max;       /* batched form: up to this many queued jobs of one batchable type (image,
                          MLP) share one launch of packed persistent kernels (default 1 = off) */
  int img_ctas_per_sm; /* batched image kernel: persistent CTAs per SM (default 4) */
  int img_tile;        /* batched image kernel tile: 0 = 32x128 (default), 1 = 16x256, 2 = 64x64 */
  int stamps;          /* 1: stage kernels write entry / exit tickets of one device counter and the
                          completion path checks every DAG edge (exit of a stage before entry of
                          its successor); violations count in set_stats_t.order_errors (test
                          invariant, default 0) */
  size_t arena_bytes;  /* serving form: 0 (default) = every job uses its slot's memory; > 0 = each
                          job's in/out/scratch is allocated at dispatch from a device arena of this
                          size (buddy blocks, 64 KiB minimum) and freed by its completion callback,
                          so jobs are admitted by free memory; slots then hold only the kernels'
                          control state and slot_bytes only bounds the largest job */
  int bind_at_submit;  /* 0 (default): UpdateGraphParams at dispatch (a dispatch thread binds the job
                          to the slot it pops); 1: at submit, as Algorithm 1 lists it: the
                          submitting thread takes a free slot if one is ready, rebinds the slot's
                          graph to the job and queues it bound, so dispatch threads only launch
                          (jobs that find no free slot are bound at dispatch); 2: as 1, and the
                          submitting thread also launches the bound job (one completion per job),
                          so an idle executor starts a job without waking a dispatch thread.  With
                          arena_bytes the job is bound at submit only if its block is free then.
                          Not with batch_max > 1. */
  int guards;          /* 1: bounds check of the stage kernels (a test instrument; compute-sanitizer
                          is not available): each job's in, out and scratch regions in its slot are
                          followed, and `in` preceded, by 256-byte guard bands that a kernel writes
                          with a pattern before the job's H2D copy and another checks after its last
                          stage kernel; a changed band sets SET_DEVERR_GUARD in the trailer and the
                          job completes with SET_EDEVICE.  Slots need kGuardBytes * 4 + 1 KiB more
                          than set_job_slot_bytes.  SET_IO_HOST (the host reads the trailer), per-job
                          graphs only (not with arena_bytes or batch_max > 1).  Default 0. */
  int sm_copies;       /* 1: a job graph's H2D and D2H steps are copy kernels (many CTAs moving 16-byte
                          words over NVLink-C2C) instead of memcpy nodes on the copy engines, which
                          pay a fixed setup per copy at these job sizes.  SET_IO_HOST only, per-job
                          graphs only (not with batch_max > 1); in / out must be page-locked host
                          memory mapped at the same address and 16-byte aligned (SET_EINVAL at
                          submit otherwise).  Default 0 (the paper's copy nodes). */
} set_config;

typedef struct {
  uint64_t submitted, completed, failed;
  uint64_t steals;          /* jobs launched by a lane other than the one they were queued on */
  uint64_t updates;         /* graph parameter updates issued (node calls) */
  uint64_t canary_errors;   /* trailers that did not match the job (should be 0) */
  double elapsed_s;         /* first submit to last completion */
  double jobs_per_s;        /* completed / elapsed_s */
  double p50_us, p99_us, max_us; /* submit -> completion callback latency */
  double mean_update_us;    /* host time of UpdateGraphParams per job */
  double mean_launch_us;    /* host time of graph launch + callback chaining per job */
  uint64_t mem_waits;       /* arena mode: dispatches that waited for free memory */
  uint64_t order_errors;    /* stamps mode: jobs whose stage order was violated (should be 0) */
  uint64_t arena_peak_bytes;/* arena mode: peak bytes allocated */
  double mean_queue_us;     /* arrival (submit) -> a dispatcher holds the job, a slot and (arena
                               mode) its device memory, and starts launching it */
  double mean_service_us;   /* launching starts -> the job's completion is handled on the
                               host: parameter updates and launch calls, device time, callback
                               delivery */
  double mean_kernel_gap_us; /* mean gap between consecutive kernels on the device timeline, from
                               the last CUPTI trace (set_trace_start / set_trace_stop) that began
                               after the last set_reset_stats; NaN when there is none */
} set_stats_t;

/* ---- sizes ---- */

/* Bytes of the H2D payload, the D2H payload (with trailer) and the device scratch of one job;
 * 0 if type or dims are invalid.  Cf. Sec. 4.1: slots are sized once and reused. */
size_t set_job_in_bytes(uint32_t type, const uint32_t dims[4]);
size_t set_job_out_bytes(uint32_t type, const uint32_t dims[4]);
size_t set_job_scratch_bytes(uint32_t type, const uint32_t dims[4]);
/* Slot bytes one job needs: in + out + scratch, each rounded up to 256 bytes. */
size_t set_job_slot_bytes(uint32_t type, const uint32_t dims[4]);

/* ---- executor (Sec. 4.2, Algorithms 1-3) ---- */

/* Defaults for every set_config field (num_streams 2, num_workers 2, ring 2, queue 4, ...). */
void set_config_default(set_config* cfg);

/* Initialization (Sec. 4.2): allocate the slot pool, create one stream per lane, instantiate
 * one graph per (slot, job type), fill W_pool with every slot and start num_workers dispatch
 * threads.  *out receives the context.  SET_ENOMEM if the pool cannot be allocated. */
set_status set_create(int num_streams, int num_workers, size_t slot_bytes, set_ctx** out);
set_status set_create_ex(const set_config* cfg, set_ctx** out);

/* Job submitter (Algorithm 1): validate, claim the next id, push to the shortest non-full lane
 * queue (lowest index on ties).  Blocks while every queue is full unless SET_F_NONBLOCK.
 * *job_id (may be NULL) receives the id echoed in the trailer.  With set_config.bind_at_submit
 * the calling thread first tries to take a free slot (and, with an arena, the job's memory block):
 * on success it rebinds the slot's graph to the job (UpdateGraphParams) and queues the slot bound
 * (1) or launches it itself (2); a launch error then completes the job with that status.  The
 * calling thread must be able to make the context's device current (it is restored after). */
set_status set_submit(set_ctx* ctx, const set_job_desc* job, uint64_t* job_id);

/* Submits n jobs in order (same rules as set_submit, one call across the boundary).
 * *first_id receives the first id; ids are consecutive only if nothing else submits
 * concurrently.  Returns at the first failure with *n_done (may be NULL) = jobs submitted. */
set_status set_submit_many(set_ctx* ctx, const set_job_desc* jobs, size_t n, uint64_t* first_id,
                           size_t* n_done);

/* Waits until every submitted job has completed (completion counter == submitted counter).
 * timeout_us < 0 waits forever.  SET_ETIMEDOUT if the time runs out. */
set_status set_wait_all(set_ctx* ctx, int64_t timeout_us);

/* Snapshot of the counters and the latency histogram (log buckets, 1/64 octave). */
set_status set_stats(set_ctx* ctx, set_stats_t* out);

/* Clears the counters, latencies and elapsed-time origin (not the job id counter). */
set_status set_reset_stats(set_ctx* ctx);

/* Drains (at most drain_timeout_ms for jobs still in flight), joins the worker threads, destroys
 * graphs, streams and (if owned) the pool. */
set_status set_destroy(set_ctx* ctx);

/* Last error text of the context (or of the calling thread's last context-less call when ctx is
 * NULL).  Valid until the next call on the same context. */
const char* set_last_error(set_ctx* ctx);

/* ---- direct launches (no graph, no executor) ---- */

/* Launches the stage kernels of one job on `stream` (a cudaStream_t, NULL = legacy default)
 * over device buffers: d_in (in_bytes), d_out (out_bytes), d_scratch (scratch_bytes, zeroed
 * once before its first use; every launch leaves it ready for the next one).  `job_id` and
 * `slot_gen` go into the trailer.  Launches that share a scratch buffer must be ordered (same
 * stream or event-chained).  Used by the single-stream baseline and for kernel timing. */
set_status set_launch_job(const set_job_desc* job, const void* d_in, void* d_out, void* d_scratch,
                          uint64_t job_id, uint32_t slot_gen, void* stream);

/* set_launch_job for a SET_JOB_SAXPY_SCAN_MAX job without any scratch buffer: for callers that
 * cannot allocate device memory (a plugin inside a process whose GPU memory belongs to another
 * allocator, or a latency-critical path where cudaMalloc would synchronise the device).  The paper
 * has no counterpart; it is an addition of this library.
 * The scratch is a file-scope static device array inside libset.so sized for n <= 16777216
 * (2^24; 65,792 bytes on every GPU that loads the library, held until process exit); larger n
 * returns SET_EINVAL with the limit in set_last_error(NULL).  d_in / d_out / stream as in
 * set_launch_job.  Allocates nothing: no cudaMalloc, no cudaFree.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.  Every call clears the
 * part of the array it uses (cudaMemsetAsync on `stream`) before its kernel.  All calls share the
 * one array: calls that overlap on the GPU (different streams without ordering) race. */
set_status set_launch_scan_static(const set_job_desc* job, const void* d_in, void* d_out, uint64_t job_id,
                                  uint32_t slot_gen, void* stream);

/* Number of kernels set_launch_job launches for this job (graph kernel nodes per job). */
int set_job_kernel_count(uint32_t type, const uint32_t dims[4], int img_fused);

/* ---- measurement helpers ---- */

/* Pinned-host <-> device copy bandwidth in GB/s for copies of `bytes` issued back to back,
 * round-robin over `streams` streams, `reps` copies in all.  dir 0 = H2D, 1 = D2H, 2 = H2D and
 * D2H together (bytes counted both ways) on the copy engines; dir 3, 4, 5 the same done by the
 * copy kernel of set_config.sm_copies.  Allocates and frees its own buffers on the current
 * device.  Used for the pipeline bound of the measured throughput. */
set_status set_copy_bandwidth(size_t bytes, int streams, int reps, int dir, double* gbs);

/* Device-timeline summary of a CUPTI activity trace (Sec. 3.2: the gaps between operations that
 * Eq. 2-4 attribute to scheduling).  Times in microseconds. */
typedef struct {
  uint64_t kernels, memcpys;   /* records traced */
  double span_us;              /* first start to last end over kernels and copies */
  double kernel_busy_us;       /* union of kernel intervals */
  double copy_busy_us;         /* union of copy intervals */
  double any_busy_us;          /* union of both */
  double idle_frac;            /* 1 - any_busy / span: the device-idle share of the span */
  double mean_kernel_gap_us;   /* mean over consecutive kernels (by start) of the idle time
                                  between the end of all earlier kernels and the next start */
  double max_kernel_gap_us;
  char top_kernel[128];        /* kernel name with the largest total time */
  uint64_t top_kernel_launches;
  double top_kernel_mean_us;   /* its mean duration */
  double top_kernel_share;     /* its share of total kernel time */
} set_trace_summary;

/* Starts recording kernels and copies of this process with CUPTI (libcupti is loaded with dlopen
 * on first use; SET_EINVAL if it cannot be found).  Tracing adds host overhead per launch: time
 * throughput without it. */
set_status set_trace_start(void);
/* Stops recording, flushes every record and fills *out. */
set_status set_trace_stop(set_trace_summary* out);

/* ---- baselines run on the same kernels (Sec. 5.1.3) ---- */

typedef enum {
  SET_BASE_SYNC = 1,        /* synchronous model: one stream, copies and kernels one by one */
  SET_BASE_BATCH_SYNC = 2   /* static batching: b streams with one graph exec each; per batch
                               update b execs, launch b, synchronise every stream, repeat */
} set_baseline_kind;

/* Runs all n jobs under a baseline model with the context's lanes, slots and graph execs (the
 * context's own dispatch threads stay idle).  Fills *out like set_stats.  Jobs with a non-zero
 * t_arrival_ns are not started before that time: SET_BASE_BATCH_SYNC then forms each batch from
 * the jobs that have arrived (at least one, at most num_streams). */
set_status set_run_baseline(set_ctx* ctx, int kind, const set_job_desc* jobs, size_t n,
                            set_stats_t* out);

/* ---- autotuner of the batched form ---- */

typedef struct {
  int batch_max;        /* jobs per launch chosen (<= the context's batch_max) */
  int img_tile;         /* image tile variant chosen */
  int img_ctas_per_sm;  /* persistent CTAs per SM chosen */
  int candidates;       /* candidates timed */
  double jobs_per_s;    /* device throughput of the packed kernels with the choice */
  double single_jobs_per_s; /* the same sample one job per launch */
} set_tune_result;

/* Times the packed kernels of `type` (image or MLP) on the sample jobs for every candidate
 * (jobs per launch 1..batch_max in powers of two; for images also tile 0..2 and 1, 2, 4, 8 CTAs
 * per SM), with CUDA events around the kernels only, and keeps the smallest jobs-per-launch within
 * 5% of the best throughput (less waiting to fill batches).  The choice applies to the context's
 * later dispatches.  The context must be idle; allocates and frees a scratch buffer. */
set_status set_autotune(set_ctx* ctx, uint32_t type, const set_job_desc* sample, size_t n, set_tune_result* out);

/* ---- serving loop (continuous batching) ---- */

#define SET_SERVE_SET 0        /* jobs go through set_submit as they arrive (the SET executor) */
#define SET_SERVE_BATCH_SYNC 1 /* the same arrivals under SET_BASE_BATCH_SYNC */

/* Request loop: job i arrives at (start + arrival_ns[i]) on CLOCK_MONOTONIC, arrival_ns ascending.
 * SET_SERVE_SET submits each job at its arrival time (t_arrival_ns set, blocking while every queue
 * is full) and waits for all; jobs that arrive while others run are admitted as slots and arena
 * memory free up and overlap on the device.  SET_SERVE_BATCH_SYNC runs the same arrivals through
 * the batch-synchronous baseline.  *out gets throughput and arrival -> completion latency. */
set_status set_serve(set_ctx* ctx, int mode, const set_job_desc* jobs, const uint64_t* arrival_ns, size_t n,
                     set_stats_t* out);

/* ---- device-side dispatch (a variant of the executor; set_dd_*) ----
 *
 * Moves dispatch and stage chaining onto the GPU.  Each lane is one stream running one graph:
 *   WHILE (loop) { fetch kernel -> SWITCH (kind) { blur kernel | scan kernel | image kernel } }.
 * set_dd_submit writes the job's descriptor (its kernel argument struct, planned on the host)
 * into a ring of the chosen lane in page-locked host memory.  The fetch kernel of each loop
 * iteration retires the jobs the previous iteration ran (a completion word each and a counter
 * written to host memory, which a thread of the context reads to complete the jobs), waits a
 * bounded time for the next descriptor, copies its arguments into the lane's device memory and
 * selects the SWITCH body.  A blur or scan descriptor takes with it the descriptors of the same
 * kind queued directly behind it (up to 8, those already published): the node runs them in one
 * launch (a cluster per blur job; a group of tiles and a scratch area per scan job).  Per job the host writes one descriptor: no graph update, no graph
 * launch and no host callback.  A lane whose fetch sees no descriptor for idle_us ends its loop; the host
 * relaunches the lane's graph when work arrives.  The paper's executor (set_create) keeps the host
 * in the loop; this variant measures the device-side alternative.
 *
 * Limits: SET_JOB_BLUR_HIST, SET_JOB_SAXPY_SCAN_MAX and SET_JOB_IMG_SOBEL_HIST (single-kernel jobs
 * whose graph node can keep one launch shape for every job of the lane: the scan node's grid
 * covers scan_max_n, the blur node's shared memory blur_max_w, and the image node's fixed grid
 * pulls the work items of any image size from the lane's ticket).  in / out must be 16-byte aligned device memory of the
 * object's GPU (checked at submit, SET_EINVAL otherwise); the kernels read and write them in
 * place.  Page-locked host buffers are refused: lane graphs whose kernels streamed them over the
 * host link faulted the GPU in testing (cause not found), so that combination is closed.  The
 * trailer's slot_gen holds the index of the lane that ran the job.  Thread safety as set_ctx. */
typedef struct set_dd set_dd; /* opaque: lanes, their graphs, rings and completion thread */

typedef struct {
  int num_lanes;         /* streams, one looping graph each (default 16) */
  int ring_depth;        /* descriptors per lane, rounded up to a power of two (default 64) */
  int device;            /* CUDA device ordinal (default 0) */
  uint32_t scan_max_n;   /* largest scan n accepted (default 65536, at most the scan limit 2^26) */
  uint32_t blur_max_w;   /* largest blur width accepted (default 256, at most the blur limit) */
  int idle_us;           /* a lane's loop ends after this long without a descriptor (default 2000) */
  int spin_us;           /* the completion thread spins this long after progress before it
                            sleeps in 5 us steps (default 50) */
  int drain_timeout_ms;  /* set_dd_destroy waits at most this long for submitted jobs (default 30000) */
} set_dd_config;

void set_dd_config_default(set_dd_config* cfg);

/* Allocates the rings (host) and lane state (device), builds and uploads each lane's graph and
 * starts the completion thread.  Lanes start idle: the first descriptor launches the loop. */
set_status set_dd_create(const set_dd_config* cfg, set_dd** out);

/* Validates the descriptor, plans the job's kernel arguments, waits for a free entry in the
 * ring of the lane with the fewest jobs in flight (lowest index on ties) unless SET_F_NONBLOCK
 * (SET_EAGAIN), publishes the entry and relaunches the lane's graph if its loop has ended. */
set_status set_dd_submit(set_dd* dd, const set_job_desc* job, uint64_t* job_id);
/* As set_submit_many.  Consecutive jobs go to one lane in groups of up to 8 (one lane choice per
 * group, the group published together, so the group's queued blur or scan jobs run as one batch);
 * a group ends before a job whose SET_F_NONBLOCK differs from its first job's, and a non-blocking
 * group publishes what fits in the ring (SET_EAGAIN once nothing fits). */
set_status set_dd_submit_many(set_dd* dd, const set_job_desc* jobs, size_t n, uint64_t* first_id, size_t* n_done);

/* As set_wait_all. */
set_status set_dd_wait_all(set_dd* dd, int64_t timeout_us);

/* Counters and latencies as set_stats (steals, updates, mem_waits, arena and stamp fields 0;
 * mean_update_us 0; mean_launch_us = host time of set_dd_submit per job; mean_queue_us and
 * mean_service_us NaN).  *graph_launches (may be NULL) gets the lane graph launches so far. */
set_status set_dd_stats(set_dd* dd, set_stats_t* out, uint64_t* graph_launches);
set_status set_dd_reset_stats(set_dd* dd);

/* Waits (drain_timeout_ms) for submitted jobs, tells every lane to end its loop, waits for the
 * lanes' streams, joins the completion thread and frees everything.  If a lane does not end,
 * its memory is left allocated (a kernel may still use it) and SET_ETIMEDOUT is returned. */
set_status set_dd_destroy(set_dd* dd);

/* Last error text of this object (or of the calling thread's last set_dd_create when NULL). */
const char* set_dd_last_error(set_dd* dd);

#ifdef __cplusplus
}
#endif

#endif /* SET_H_ */
