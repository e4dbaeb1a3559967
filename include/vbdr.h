/*
 * vbdr.h -- C ABI of the GB300 (sm_103a) VBDR library.
 *
 * VBDR ("virtual bit distance recorder", Xu, arXiv 1810.13132) estimates the
 * cardinality of many hosts under a sliding window of k time slices.  Every
 * host aip owns a virtual vector of g = 2^b bit distance recorders (BDRs)
 * drawn from one shared pool BDRP of Z physical BDRs (Sec. 4.1).  A BDR is a
 * vector of w-bit distance recorders (DRs), one per LBP1 value 1..R: a DR
 * holds how many slices ago its LBP1 value was recorded, saturating at
 * 2^w - 1, and is active while it is below k (Sec. 3).
 *
 * Per time slice t the caller
 *   1. streams the slice's (aip, bip) pairs through vbdr_scan_slice (one or
 *      more calls; Alg. 7 for the gfast layout, Alg. 9 for gsmall),
 *   2. closes the slice with vbdr_slide (Alg. 6 for gfast; Alg. 8 for
 *      gsmall) which also extracts every BDR's register (Alg. 2) and the
 *      pool-wide sums used to remove sharing noise,
 *   3. asks for estimates with vbdr_estimate (Alg. 3 + Alg. 5 + the virtual
 *      register sharing HyperLogLog estimator), which cover the window
 *      W(t-k+1, k) of the last k closed slices (fewer at start-up).
 *
 * Conventions shared by every entry point
 *   - Return value: VBDR_OK (0) or a negative vbdr_status.  A CUDA error
 *     is sticky: the handle then answers VBDR_ECUDA to every later call
 *     except vbdr_destroy.
 *   - "stream" is a cudaStream_t passed as void*; NULL is the legacy default
 *     stream.  Calls are asynchronous and ordered on that stream; a device
 *     buffer passed in must stay valid until the stream has passed the call.
 *   - d_* pointers are device memory (or memory the GPU can address); h_*
 *     pointers are host memory.  The caller owns every buffer it passes in;
 *     the handle owns its state and frees it in vbdr_destroy.
 *   - A handle is not thread-safe: one host thread at a time per handle.
 *     Different handles are independent and may run on different streams.
 *   - The library allocates only in vbdr_create (and on the first host-buffer
 *     call, see vbdr_scan_slice_host).
 */
#ifndef VBDR_H_
#define VBDR_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define VBDR_API __attribute__((visibility("default")))
#else
#define VBDR_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vbdr *vbdr_t;

typedef enum {
  VBDR_OK = 0,
  VBDR_EINVAL = -1,   /* bad argument: NULL, misaligned, out of range      */
  VBDR_ENOMEM = -2,   /* device or host allocation failed                  */
  VBDR_ECUDA = -3,    /* a CUDA call failed; the handle is now unusable    */
  VBDR_ERANGE = -4,   /* a size exceeds the handle's capacity              */
  VBDR_EORDER = -5,   /* call out of order (estimate before first slide)   */
  VBDR_ETIMEOUT = -6  /* a bounded device wait expired                     */
} vbdr_status;

/* BDR layouts of Sec. 4.2 / Table 1.
 *   VBDR_GFAST : DRV plus the bsLBP1 bit string; the scan only ORs one bit
 *                (Alg. 7), the slide folds the highest set bit (Alg. 6).
 *   VBDR_GSMALL: DRV only; the scan zeroes a DR in place (Alg. 9), the slide
 *                ages every DR (Alg. 8).  Smaller state, random RMW of the
 *                DRV during the scan.
 *   VBDR_SERIAL: DRV plus one nowLBP1 byte (Alg. 1 / 4): the scan raises
 *                nowLBP1 to the pair's LBP1 with a byte-wise atomic max (the
 *                race of Sec. 4.2 cannot lose the larger value), the slide
 *                folds it like Alg. 6.  Same DRV as gfast after every slide.*/
typedef enum { VBDR_GFAST = 0, VBDR_GSMALL = 1, VBDR_SERIAL = 2 } vbdr_layout;

typedef struct {
  uint32_t k;          /* slices per window, 1..255                         */
  uint32_t log2_g;     /* b of every host when group_rule = 0, 1..16        */
  uint32_t log2_g_min; /* smallest b in use (0 = log2_g); R = 32 - b_min    */
  uint32_t group_rule; /* 0: every host has b = log2_g;
                          1: host aip has b = log2_g_min + (aip >> 30),
                             i.e. four groups g = 2^b_min .. 2^(b_min+3);
                             requires b_min + 3 <= 9                        */
  uint32_t layout;     /* vbdr_layout                                       */
  uint32_t reserved;   /* must be 0                                         */
  uint64_t num_bdr;    /* Z, physical BDRs; must exceed the largest g,
                          at most 2^32 - 1 (the exact pool sum
                          sum_j 2^(32 - reg_j) <= Z 2^32 must fit 64 bits) */
  uint64_t seed;       /* hash seed A0 (Sec. 4.1); A1 is derived from it    */
} vbdr_config;

/* Create a handle and its device-resident state on the current CUDA device
 * (InitDR on every DR: all DRs start at 2^w - 1, w = ceil(log2(k+1))).
 * Device memory: DRV ceil(R / floor(32/w)) * 4 B per BDR, plus 4 B bsLBP1
 * per BDR for gfast, plus 1 B register per BDR.  Errors: VBDR_EINVAL,
 * VBDR_ENOMEM, VBDR_ECUDA.  *out is NULL on failure. */
VBDR_API int vbdr_create(const vbdr_config *cfg, vbdr_t *out);

/* Free all state.  Accepts NULL.  Synchronises the device first. */
VBDR_API int vbdr_destroy(vbdr_t h);

/* Scan n pairs of the current slice (Sec. 4.2, Alg. 7 for gfast, Alg. 9 for
 * gsmall; per pair the steps of Alg. 4: hash bip with A1, virtual index =
 * its left b bits, LBP1 of the rest, physical BDR by Alg. 3).
 * d_pairs: 2n uint32 on the device, array-of-structs (aip, bip), 16-byte
 * aligned.  n = 0 is a no-op.  May be called several times per slice; the
 * result does not depend on the order or split of the pairs.
 * Errors: VBDR_EINVAL (NULL with n > 0, misaligned), VBDR_ECUDA. */
VBDR_API int vbdr_scan_slice(vbdr_t h, const uint32_t *d_pairs, uint64_t n,
                    void *stream);

/* The same as vbdr_scan_slice for pairs in HOST memory: the pairs are copied
 * to the device in chunks through a staging ring owned by the handle (allocated
 * on the first call), overlapped with the scan of the previous chunk.
 * h_pairs should be pinned (cudaHostAlloc / cudaHostRegister) for full copy
 * speed; pageable memory works but is slower.  The call returns once every
 * chunk is enqueued; h_pairs must stay valid until the stream has passed it.
 * The copies (on the handle's own copy stream) do not wait for work enqueued
 * earlier on the stream, only the scans do: h_pairs must already hold the
 * pairs when the call is made, and the copies overlap earlier slides and
 * estimates on the stream.
 * Errors: as vbdr_scan_slice, plus VBDR_ENOMEM. */
VBDR_API int vbdr_scan_slice_host(vbdr_t h, const uint32_t *h_pairs, uint64_t n,
                         void *stream);

/* vbdr_scan_slice with the pair count read from device memory when the
 * kernel runs: min(*d_n, max_n) pairs of d_pairs are scanned (d_n: one
 * uint64 on the device, 8-byte aligned).  A CUDA graph captured around this
 * call serves slices of any size up to max_n.  Errors: as vbdr_scan_slice. */
VBDR_API int vbdr_scan_slice_devn(vbdr_t h, const uint32_t *d_pairs, const uint64_t *d_n,
                                  uint64_t max_n, void *stream);

/* Close the current slice (Sec. 3 and 4.2).
 *   gfast : every BDR slides all DRs, sets the DR of the highest set bit of
 *           bsLBP1 (Alg. 6) and clears bsLBP1; then its register is read
 *           (Alg. 2).
 *   gsmall: every BDR's register is read (Alg. 2, window just closed), then
 *           all DRs slide (Alg. 8 for the next slice).
 * Also computes the pool sums S_Z = sum_j 2^(32 - reg_j) and V_Z = #{reg_j
 * = 0} over all Z registers.  Errors: VBDR_ECUDA. */
VBDR_API int vbdr_slide(vbdr_t h, void *stream);

/* Estimate the cardinality of n_hosts hosts over the window of the last k
 * closed slices (Definition 1, Alg. 5 and the virtual register sharing
 * estimator n = Z g/(Z-g) (n_g/g - n_Z/Z) with HyperLogLog estimates n_g of
 * the host's g registers and n_Z of the pool, both with small-range linear
 * counting; clamped at 0).  Harmonic sums are exact integers; the formula
 * is evaluated in FP64 and rounded to FP32.
 * d_aips: n_hosts uint32 host addresses (device); d_out: n_hosts float
 * (device).  n_hosts = 0 is a no-op.
 * Errors: VBDR_EINVAL, VBDR_EORDER (no slide yet), VBDR_ECUDA. */
VBDR_API int vbdr_estimate(vbdr_t h, const uint32_t *d_aips, uint64_t n_hosts,
                  float *d_out, void *stream);

/* Estimators the BDR pool can serve besides HyperLogLog (Sec. 4.1 notes
 * PCSA and LogLog counting), each with the same virtual-sharing noise
 * removal n = Z g/(Z-g) (n_g/g - n_Z/Z), clamped at 0, in FP64:
 *   VBDR_EST_HLL   : vbdr_estimate.
 *   VBDR_EST_LOGLOG: n_m = alpha_m m 2^(sum M / m) over the registers M
 *                    (Alg. 5's getSumLBP1 is the sum), alpha_m =
 *                    (Gamma(-1/m) (1 - 2^(1/m)) / ln 2)^(-m) (Durand &
 *                    Flajolet 2003).  Any layout.
 *   VBDR_EST_PCSA  : n_m = (m / 0.77351) 2^(sum R / m) (Flajolet & Martin
 *                    1985), R of a BDR = the number of active DRs from
 *                    LBP1 1 up to the first inactive one, i.e. the lowest
 *                    unset position of the window bitmap.  Needs a bitmap of
 *                    every LBP1 seen, which only gsmall's Alg. 9 records:
 *                    gsmall only (its slide stores R for every BDR). */
typedef enum { VBDR_EST_HLL = 0, VBDR_EST_LOGLOG = 1, VBDR_EST_PCSA = 2 } vbdr_estimator;

/* vbdr_estimate with the estimator of the given vbdr_estimator.
 * Errors: as vbdr_estimate; VBDR_EINVAL also for an unknown estimator or
 * VBDR_EST_PCSA on a layout other than VBDR_GSMALL. */
VBDR_API int vbdr_estimate_alt(vbdr_t h, const uint32_t *d_aips, uint64_t n_hosts, float *d_out,
                               int estimator, void *stream);

/* vbdr_estimate for HOST buffers: h_aips is copied in, h_out is written back
 * on the stream (valid once the stream has passed the call).  Uses a staging
 * buffer owned by the handle, grown as needed.  Errors: as vbdr_estimate,
 * plus VBDR_ENOMEM. */
VBDR_API int vbdr_estimate_host(vbdr_t h, const uint32_t *h_aips, uint64_t n_hosts,
                       float *h_out, void *stream);

/* Estimate plans.  The host-to-register map of Alg. 3 (host aip, virtual
 * index i -> physical BDR) depends only on the host address, i and the
 * handle's configuration, so a host list that is estimated after every slide
 * can have it computed once.  A plan holds it grouped by 32 KiB register
 * chunk; vbdr_estimate_planned then streams the register array through
 * shared memory once per block of hosts instead of gathering H g random
 * bytes.  The estimates equal vbdr_estimate's for the same hosts, bit for
 * bit (same exact integer sums, same FP64 formula).
 * Plans are valid for every handle with the same Z, log2_g, log2_g_min,
 * group_rule and seed on the same device; they do not depend on the state.
 * Memory: 4 bytes per virtual register of the list (H g in all, plus at most
 * 3 per register chunk and block of hosts of padding), 4 bytes per host and
 * 8 bytes per (block, chunk) pair. */
typedef struct vbdr_plan *vbdr_plan_t;

/* Build the plan of n_hosts hosts (d_aips: uint32 host addresses, device,
 * 4-byte aligned; copied, so the buffer may be reused after the call).
 * Synchronises the stream (the group sizes are read back to lay out the
 * plan).  n_hosts = 0 gives an empty plan.
 * Errors: VBDR_EINVAL (NULL or misaligned), VBDR_ERANGE (Z > 2^28),
 * VBDR_ENOMEM, VBDR_ECUDA. */
VBDR_API int vbdr_plan_create(vbdr_t h, const uint32_t *d_aips, uint64_t n_hosts,
                              vbdr_plan_t *out, void *stream);
/* Free a plan (NULL is accepted).  No call that uses it may be in flight. */
VBDR_API int vbdr_plan_destroy(vbdr_plan_t p);
/* Hosts, stored entries (including padding) and device bytes of a plan;
 * any output pointer may be NULL.  Errors: VBDR_EINVAL. */
VBDR_API int vbdr_plan_info(vbdr_plan_t p, uint64_t *n_hosts, uint64_t *n_entries,
                            uint64_t *device_bytes);
/* Synchronous check of the plan's device error word: VBDR_ETIMEOUT if a
 * bounded wait inside an earlier vbdr_estimate_planned expired (that call's
 * outputs for the affected block of hosts are NaN), else VBDR_OK. */
VBDR_API int vbdr_plan_status(vbdr_plan_t p);

/* vbdr_estimate for the plan's hosts, in the order given at vbdr_plan_create:
 * d_out[i] (device, n_hosts floats, 4-byte aligned) is host i's estimate.
 * Errors: VBDR_EINVAL (NULL, misaligned, plan built for another
 * configuration or device), VBDR_EORDER (no slide yet), VBDR_ECUDA. */
VBDR_API int vbdr_estimate_planned(vbdr_t h, vbdr_plan_t p, float *d_out, void *stream);

/* vbdr_estimate_planned with the compact learned correction applied in the
 * same kernel (not in the paper; a trained correction of the plain vHLL
 * estimate against sharing noise).  Per host the kernel also counts the
 * virtual registers holding 0, 1, 2 and 3 (n_0 = V .. n_3) and forms ten
 * inputs: n_0/g .. n_3/g, log2 g / 16, ln(1 + n_plain) / 16, ln(1 + n_g) / 16
 * (n_g the host's raw or linear-counting estimate before noise removal),
 * ln(1 + n_Z / Z), V_Z / Z and V / g; a network of two layers of 16
 * tanh-form GELUs gives delta, and the host's estimate is
 * max(0, exp(ln(1 + n_plain) + delta) - 1), or n_plain itself where
 * n_plain > nmax.  FP32 arithmetic after the FP64 plain estimate.
 * h_theta: HOST memory, 465 FP32 values, copied into the launch during the
 * call (the caller may reuse the buffer at once): W1 [16][10] row-major,
 * b1 [16], W2 [16][16], b2 [16], w3 [16], b3.  nmax: the largest plain
 * estimate the network was trained on.  d_out as in vbdr_estimate_planned.
 * Requires every g <= 512.  Runs two kernels: the planned estimate, which
 * also writes a 16-byte record per host into a buffer owned by the handle
 * (grown on first use after synchronising the stream, so make the first
 * call outside any stream capture), and the network over the records.
 * Errors: as vbdr_estimate_planned, plus VBDR_ERANGE (g above 512) and
 * VBDR_ENOMEM. */
VBDR_API int vbdr_estimate_planned_compact(vbdr_t h, vbdr_plan_t p, const float *h_theta,
                                           float nmax, float *d_out, void *stream);

/* A plan as vbdr_plan_create builds it, with blocks of at most 3300 hosts:
 * what vbdr_estimate_learned_planned needs (its per-host register
 * histograms share a block's shared memory); vbdr_estimate_planned accepts
 * it too.  Errors: as vbdr_plan_create. */
VBDR_API int vbdr_plan_create_learned(vbdr_t h, const uint32_t *d_aips, uint64_t n,
                                      vbdr_plan_t *out, void *stream);

/* vbdr_estimate_planned with the estimates written to HOST memory h_out
 * (valid once the stream has passed the call), through a device buffer owned
 * by the handle.  Errors: as vbdr_estimate_planned, plus VBDR_ENOMEM. */
VBDR_API int vbdr_estimate_planned_host(vbdr_t h, vbdr_plan_t p, float *h_out, void *stream);

/* Estimates for n_hosts hosts computed straight from a register array that
 * the caller already holds in device memory, without allocating anything.
 * The paper has no counterpart of this call; it serves callers that cannot
 * call cudaMalloc where they need an estimate -- for instance a process whose
 * device memory is all reserved at start-up by a framework's own allocator,
 * or a latency-critical loop that forbids allocation once it runs -- and so
 * cannot create a handle.
 * d_reg: num_bdr uint8 registers (one per physical BDR, as written by
 * vbdr_slide: the largest active LBP1, 0 if none; a value above 32 is read
 * as 32); log2_g: b of every host,
 * 1..9; seed: the A0 the registers were built with; d_aips / d_out: as in
 * vbdr_estimate.  The result equals vbdr_estimate on a handle whose registers
 * are d_reg (same FP64 formula, rounded to FP32).
 * Working memory: a fixed array of about 12.4 KiB compiled into the library
 * (seed table for g <= 512, ln table, pool-sum accumulators); every GPU that
 * loads the library holds it until the process exits.  The first call on
 * each device, with that device current, looks up the array's device address
 * (cudaGetSymbolAddress) and caches it, so make that first call before any
 * stream capture.  Each call rebuilds the tables for its seed and clears the
 * accumulators; all calls share the one array, so calls whose work overlaps
 * on the GPU (other streams, other host threads) race and must be
 * serialised by the caller.  The cached address belongs to the CUDA context
 * it was looked up in: after cudaDeviceReset on that device the library's
 * module is loaded again elsewhere and the cached address is stale, so do
 * not call this function after a device reset in the same process.  No
 * cudaMalloc, cudaFree or allocating library routine is called.
 * Errors: VBDR_ERANGE (log2_g > 9), VBDR_EINVAL (NULL or misaligned pointer,
 * log2_g < 1, num_bdr not in (2^log2_g, 2^32 - 1]), VBDR_ECUDA. */
VBDR_API int vbdr_estimate_registers_noalloc(const uint8_t *d_reg, uint64_t num_bdr,
                                             uint32_t log2_g, uint64_t seed,
                                             const uint32_t *d_aips, uint64_t n_hosts,
                                             float *d_out, void *stream);

/* Scan kernels.  VBDR_SCAN_DIRECT (the default): each pair's update word
 * is tested with one cached load and changed with one atomic only when the
 * update changes it (Alg. 7 / Alg. 9 / Alg. 4).  VBDR_SCAN_BUCKETED: for
 * slices of at least 2^18 pairs, the pairs are routed as 4-byte records to
 * the 2^16-BDR tile of the pool that owns them and every tile applies its
 * records in shared memory, writing the state once per scan call (gfast
 * and gsmall only, g <= 512, Z <= 2^27).  Both give the same state bit for
 * bit; the direct kernel is faster on this GPU (the bucketed one is kept
 * for measurement).  Selecting the bucketed scan allocates its buffers once
 * (about 64 MiB for a 2^24 pool) after synchronising the device, so select
 * it before any stream capture.  Errors: VBDR_EINVAL (unknown mode, or
 * bucketed on a layout or size it does not serve), VBDR_ENOMEM. */
#define VBDR_SCAN_DIRECT 0
#define VBDR_SCAN_BUCKETED 1
VBDR_API int vbdr_set_scan_mode(vbdr_t h, int mode);

/* ---- several GPUs --------------------------------------------------------
 * The paper's scan is data parallel over pairs and its slide over BDRs
 * (Sec. 4.2): every update ORs a bsLBP1 bit (Alg. 7), zeroes a DR (Alg. 9)
 * or raises nowLBP1 (Alg. 4), all commutative and idempotent.  A pool spread
 * over ranks therefore needs only these exchanges, which the caller performs
 * with any transport (NCCL, ...); the calls below read and write device
 * buffers of one handle on its own device.
 *   Pair-sharded replicas: every rank scans its share of a slice into a full
 *   replica, the ranks exchange their slice states and merge them with
 *   vbdr_merge_slice_state before the slide, and every rank slides the same
 *   merged state.
 *   Pool-partitioned: rank r owns BDRs [r Zr, (r+1) Zr), Zr = ceil(Z / ranks);
 *   every rank turns its pairs into records with vbdr_route_records, the
 *   ranks exchange the groups (all-to-all), each applies what it received
 *   with vbdr_apply_records and slides; the byte-wise maximum of the ranks'
 *   register arrays (every register outside a rank's range is 0 there) is
 *   the pool's, installed on every rank with vbdr_set_registers. */

/* Device pointers of the handle's state, owned by the handle (valid until
 * vbdr_destroy; read them only between calls that write them):
 * d_slice_state / slice_words: the state a scan updates, as 32-bit words --
 * bsLBP1 [Z] (gfast), the DRV planes [P][Zs] (gsmall), nowLBP1 bytes [Zs] as
 * Zs/4 words (serial); d_reg: the Z registers of the last slide; d_pcsa: the
 * Z PCSA statistics (gsmall, else NULL).  Any output may be NULL.
 * Errors: VBDR_EINVAL (NULL handle). */
VBDR_API int vbdr_state_pointers(vbdr_t h, uint32_t **d_slice_state, uint64_t *slice_words,
                                 uint8_t **d_reg, uint8_t **d_pcsa);

/* Hash n pairs (d_pairs as in vbdr_scan_slice, 4-byte aligned suffices) into
 * records pidx << 5 | (LBP1 - 1) (Alg. 4 and Alg. 3), grouped by the rank
 * owning pidx: group r is d_recs[r cap, r cap + min(d_fill[r], cap)), in no
 * particular order.  d_recs: device, n_ranks * cap uint32; d_fill: device,
 * n_ranks uint64 (8-byte aligned), set by the call; d_fill[r] > cap means
 * group r overflowed and records were dropped -- size cap for the worst
 * case (cap = n always suffices).  Requires Z <= 2^27 and every g <= 512.
 * The state is not changed.  Errors: VBDR_EINVAL (NULL or misaligned
 * pointer, n_ranks not in 1..256, Z > 2^27), VBDR_ERANGE (g above 512),
 * VBDR_ECUDA. */
VBDR_API int vbdr_route_records(vbdr_t h, const uint32_t *d_pairs, uint64_t n, uint32_t n_ranks,
                                uint32_t *d_recs, uint64_t cap, uint64_t *d_fill, void *stream);

/* Apply n records pidx << 5 | (LBP1 - 1) (from vbdr_route_records, on any
 * rank) to the handle's slice state: the same update the scan of their pairs
 * makes (Alg. 7, Alg. 9 or Alg. 4).  d_recs: device, 4-byte aligned.
 * Errors: VBDR_EINVAL (NULL or misaligned, Z > 2^27), VBDR_ECUDA. */
VBDR_API int vbdr_apply_records(vbdr_t h, const uint32_t *d_recs, uint64_t n, void *stream);

/* Merge another replica's slice state (same configuration; d_other: device,
 * slice_words words laid out as vbdr_state_pointers gives them) into this
 * handle's: OR of bsLBP1 (gfast), field-wise minimum of the DRs (gsmall),
 * maximum of nowLBP1 (serial).  Errors: VBDR_EINVAL, VBDR_ECUDA. */
VBDR_API int vbdr_merge_slice_state(vbdr_t h, const uint32_t *d_other, void *stream);

/* Install Z registers (d_reg, device) and, for gsmall, the Z PCSA statistics
 * (d_pcsa, device, may be NULL) as the registers of the last slide, and
 * recompute the pool sums the estimators read (Sec. 4.1's noise term).
 * The next slide overwrites them.  Errors: VBDR_EINVAL (NULL d_reg, d_pcsa
 * on a layout without PCSA statistics), VBDR_ECUDA. */
VBDR_API int vbdr_set_registers(vbdr_t h, const uint8_t *d_reg, const uint8_t *d_pcsa,
                                void *stream);

/* Register-level state for workloads too large to scan (batched estimation
 * over millions of hosts): the register array becomes, for every physical
 * BDR, the largest value among the virtual registers that Alg. 3 maps onto
 * it -- host d_aips[h]'s virtual index i goes to BDR getPhyIdx(aip, i) -- and
 * 0 where none maps; the pool sums are recomputed and the handle becomes
 * ready for vbdr_estimate.  d_vregs[d_offsets[h] + i], i < g(aip), holds host
 * h's i-th virtual register (uint8, at most 32 - b).  The DRV is not touched:
 * the next vbdr_slide recomputes the registers from it.
 * Errors: VBDR_EINVAL, VBDR_ECUDA. */
VBDR_API int vbdr_load_virtual_registers(vbdr_t h, const uint32_t *d_aips,
                                         const uint64_t *d_offsets, uint64_t n_hosts,
                                         const uint8_t *d_vregs, void *stream);

/* Launch shape of vbdr_estimate: lanes cooperating on one host (8, 16, 32)
 * and threads per block (32..512, multiple of 32).  The estimate is one
 * persistent launch (one wave of blocks, grid-stride over batches of 32
 * hosts) whatever the shape; the shape changes only the speed, never the
 * result.  Default 32 lanes, 256 threads.  Errors: VBDR_EINVAL. */
VBDR_API int vbdr_set_estimate_launch(vbdr_t h, uint32_t lanes, uint32_t threads);

/* Autotuner of the estimate launch shape (Sec. 4.2's parallel estimation,
 * batched over hosts of mixed g): times every candidate shape on these hosts
 * (one warm-up and two timed launches each, writing d_out), keeps the fastest
 * for later vbdr_estimate calls and reports it in *lanes / *threads (either
 * may be NULL).  Synchronises the stream.
 * Errors: VBDR_EINVAL, VBDR_EORDER, VBDR_ECUDA. */
VBDR_API int vbdr_autotune_estimate(vbdr_t h, const uint32_t *d_aips, uint64_t n_hosts,
                                    float *d_out, uint32_t *lanes, uint32_t *threads,
                                    void *stream);

/* ---- learned correction (not in the paper) ----
 * A 2 x 64 GELU MLP maps a host's feature vector to delta, a correction of
 * the plain estimate in log space: n = exp(ln(1 + n_plain) + delta) - 1.
 * Features (80 inputs): x[v] = #{virtual registers of value v} / g for
 * v = 0..63, x[64] = b/16, x[65] = ln(1 + n_plain)/16, x[66] = ln(1 + n_g)/16
 * (the host's own HLL estimate), x[67] = ln(1 + n_Z/Z), x[68] = V_Z/Z,
 * x[69] = V/g, x[70..79] = 0.  Registers never exceed 31, so bins 32..63 are
 * always 0; device feature matrices carry the 48 live inputs per row as BF16:
 * x[0..31] then x[64..79].  Weights BF16, accumulation FP32 (tensor cores),
 * FP32 master parameters trained by AdamW on the GPU.  Parameters travel as
 * a flat FP32 vector: W1 [64][80] row-major, b1 [64], W2 [64][64], b2 [64],
 * w3 [64], b3 [1] (vbdr_mlp_num_params() floats).  Hosts whose plain
 * estimate exceeds nmax keep the plain estimate (the range the network was
 * trained on). */
typedef struct vbdr_mlp *vbdr_mlp_t;

VBDR_API int vbdr_mlp_num_params(void);

/* New network on the current device, weights drawn from a seeded uniform
 * (He) initialisation, biases 0, nmax = +inf.  Errors: VBDR_EINVAL,
 * VBDR_ENOMEM. */
VBDR_API int vbdr_mlp_create(uint64_t seed, vbdr_mlp_t *out);
VBDR_API int vbdr_mlp_destroy(vbdr_mlp_t m);

/* Replace / read the FP32 parameters (host buffers of vbdr_mlp_num_params()
 * floats) and nmax.  set resets the optimizer state.  Synchronous. */
VBDR_API int vbdr_mlp_set_params(vbdr_mlp_t m, const float *h_params, float nmax);
VBDR_API int vbdr_mlp_get_params(vbdr_mlp_t m, float *h_params, float *nmax);

/* Train on n samples: d_X BF16 [n][48] live features (device), d_y FP32 [n]
 * targets delta* = ln(1 + c) - ln(1 + n_plain) (device); loss = mean squared
 * error; `epochs` passes of contiguous batches of `batch` samples (shuffle
 * the set beforehand), AdamW (beta 0.9/0.999, eps 1e-8) with learning rate lr
 * and decoupled weight decay on the weight matrices.  h_epoch_loss (host,
 * `epochs` floats, may be NULL) receives each epoch's mean loss.  Synchronises
 * the stream once per epoch when h_epoch_loss is given.
 * Errors: VBDR_EINVAL, VBDR_ECUDA. */
VBDR_API int vbdr_mlp_train(vbdr_mlp_t m, const uint16_t *d_X, const float *d_y, uint64_t n,
                            uint32_t epochs, uint32_t batch, float lr, float weight_decay,
                            uint64_t shuffle_seed, float *h_epoch_loss, void *stream);

/* Gradient of the mean squared error over n samples at the current
 * parameters (h_grad: vbdr_mlp_num_params() floats, host) and the loss.
 * Synchronous.  For checking the backward kernels. */
VBDR_API int vbdr_mlp_gradient(vbdr_mlp_t m, const uint16_t *d_X, const float *d_y, uint64_t n,
                               float *h_grad, float *h_loss, void *stream);

/* delta for n feature rows (d_X BF16 [n][48], 16-byte aligned; d_delta FP32
 * [n]; both device).  Errors: VBDR_EINVAL (NULL or misaligned), VBDR_ECUDA. */
VBDR_API int vbdr_mlp_forward(vbdr_mlp_t m, const uint16_t *d_X, uint64_t n, float *d_delta,
                              void *stream);

/* Feature rows of n hosts from the handle's registers (d_X BF16 [n][48],
 * device, 16-byte aligned) and their plain estimates (d_plain FP32 [n],
 * device, may be NULL).  The histogram bins count in 16-bit fields, so every
 * host's g must be at most 512 (the learned correction is trained on
 * g = 256).  Errors: as vbdr_estimate, plus VBDR_ERANGE (largest g of the
 * handle above 512) and VBDR_EINVAL (d_X not 16-byte aligned). */
VBDR_API int vbdr_features(vbdr_t h, const uint32_t *d_aips, uint64_t n_hosts, uint16_t *d_X,
                           float *d_plain, void *stream);

/* vbdr_estimate with the learned correction fused into the same kernel:
 * the gather also builds each host's register histogram, the MLP runs on the
 * tensor cores per batch of 32 hosts, and d_out receives the corrected
 * estimate (the plain one where n_plain > nmax).  Errors: as vbdr_estimate,
 * plus VBDR_ERANGE (largest g of the handle above 512, as vbdr_features). */
VBDR_API int vbdr_estimate_learned(vbdr_t h, vbdr_mlp_t m, const uint32_t *d_aips,
                                   uint64_t n_hosts, float *d_out, void *stream);

/* vbdr_estimate_learned for the hosts of a plan made by
 * vbdr_plan_create_learned: the same feature rows and the same corrected
 * estimates, bit for bit, with the registers read chunk by chunk through the
 * plan instead of gathered (Alg. 5 with Alg. 3 as in vbdr_estimate_planned).
 * d_out: device, n_hosts floats, 4-byte aligned, plan order.  Errors:
 * VBDR_EINVAL (NULL, misaligned, plan of another configuration or built by
 * vbdr_plan_create), VBDR_ERANGE (a g above 512), VBDR_EORDER, VBDR_ENOMEM,
 * VBDR_ECUDA; a bounded wait that expired shows in vbdr_plan_status. */
VBDR_API int vbdr_estimate_learned_planned(vbdr_t h, vbdr_mlp_t m, vbdr_plan_t p, float *d_out,
                                           void *stream);

/* ---- streaming service ----
 * A server runs many VBDR instances ("tenants", e.g. one per monitored
 * link) on one GPU.  Each tenant keeps its BDR pool on the device for its
 * whole life and owns a copy stream, a compute stream and two captured CUDA
 * graphs (one per staging buffer), each holding the full per-slice path:
 * scan (slice size read from device memory) -> slide -> estimate of the
 * tenant's hosts (plain, or with the learned correction) -> copy of the
 * estimates to pinned host memory.  A tenant's slices run in order, two at
 * most in flight; tenants run concurrently and overlap on the device.
 * Admission: a tenant's device footprint (vbdr_server_tenant_bytes) must fit
 * in the server's budget next to the admitted ones; otherwise vbdr_server_open
 * waits, bounded by its timeout, until tenants close and free memory. */
typedef struct vbdr_server *vbdr_server_t;
typedef struct {
  uint64_t device_budget_bytes; /* device memory all tenants may hold together */
  uint32_t max_tenants;         /* 1..1024 */
  uint32_t reserved;            /* must be 0 */
} vbdr_server_config;

VBDR_API int vbdr_server_create(const vbdr_server_config *cfg, vbdr_server_t *out);
/* Closes every tenant.  Accepts NULL. */
VBDR_API int vbdr_server_destroy(vbdr_server_t s);

/* Device bytes a tenant holds (state, tables, two staging slots, hosts). */
VBDR_API uint64_t vbdr_server_tenant_bytes(const vbdr_config *cfg, uint64_t max_pairs,
                                           uint64_t n_hosts);

/* Admit a tenant with handle configuration cfg, slices of up to max_pairs
 * pairs and the n_hosts hosts h_aips (host memory, copied) to estimate after
 * every slice; mlp (may be NULL) adds the learned correction.  Waits up to
 * timeout_ms for room.  On the fresh state it closes one empty slice (which
 * changes nothing) before capturing the graphs.
 * Errors: VBDR_EINVAL, VBDR_ERANGE (larger than the whole budget),
 * VBDR_ETIMEOUT, VBDR_ENOMEM, VBDR_ECUDA. */
VBDR_API int vbdr_server_open(vbdr_server_t s, const vbdr_config *cfg, uint64_t max_pairs,
                              const uint32_t *h_aips, uint64_t n_hosts, vbdr_mlp_t mlp,
                              uint32_t timeout_ms, uint32_t *tenant);
/* Release a tenant's memory (after its work finishes) and wake waiters. */
VBDR_API int vbdr_server_close(vbdr_server_t s, uint32_t tenant);

/* Enqueue one slice of n pairs (h_pairs: host memory, pinned for full copy
 * speed, valid until the slice's wait returns).  Returns a ticket.
 * Errors: VBDR_ERANGE (n > max_pairs), VBDR_EORDER (two slices of this tenant
 * already in flight: wait for one first), VBDR_EINVAL, VBDR_ECUDA. */
VBDR_API int vbdr_server_submit(vbdr_server_t s, uint32_t tenant, const uint32_t *h_pairs,
                                uint64_t n, uint64_t *ticket);

/* Wait (host-side polling, bounded by timeout_ms) for a ticket; copy the
 * slice's estimates into h_out (n_hosts floats, may be NULL).  device_ms: the
 * graph's execution time; e2e_ms: submit to completion.  Either may be NULL.
 * Errors: VBDR_EINVAL, VBDR_ETIMEOUT, VBDR_ECUDA. */
VBDR_API int vbdr_server_wait(vbdr_server_t s, uint32_t tenant, uint64_t ticket, float *h_out,
                              uint32_t timeout_ms, float *device_ms, float *e2e_ms);

/* Device bytes and tenants currently admitted. */
VBDR_API int vbdr_server_in_use(vbdr_server_t s, uint64_t *bytes, uint32_t *tenants);

/* The handle that holds a tenant's BDR state (owned by the server: never
 * destroy it), for inspection with vbdr_copy_state / vbdr_copy_pool_sums /
 * vbdr_save once every submitted slice of the tenant has been waited for
 * (the state then reflects all of them; between submit and wait it is in
 * flight on the tenant's streams).  Valid until vbdr_server_close of the
 * tenant.  Errors: VBDR_EINVAL (no such tenant, NULL out). */
VBDR_API int vbdr_server_tenant_handle(vbdr_server_t s, uint32_t tenant, vbdr_t *out);

/* ---- checkpoint / resume ----
 * The complete state of a handle -- configuration, DRV, the slice state
 * (bsLBP1 / nowLBP1 of the current, unclosed slice), registers, PCSA
 * statistics (gsmall) and all pool sums of the last slide -- as one host
 * buffer: an 80-byte header ("VBDRCKP2", configuration, buffer sizes)
 * followed by the raw device buffers.  A handle created with the same
 * configuration that loads it continues exactly as the saved one would have
 * (bit for bit).  Both calls synchronise the stream.
 * save: VBDR_ERANGE if cap < vbdr_state_bytes.  load: VBDR_EINVAL if the
 * buffer is short, was saved with another configuration or by another
 * format version. */
VBDR_API int vbdr_state_bytes(vbdr_t h, uint64_t *bytes);
VBDR_API int vbdr_save(vbdr_t h, void *h_buf, uint64_t cap, void *stream);
VBDR_API int vbdr_load(vbdr_t h, const void *h_buf, uint64_t len, void *stream);

/* ---- inspection (tests, debugging); these synchronise the stream ---- */

/* Derived sizes: R (DRs per BDR), w (DR bits), words (32-bit DRV words per
 * BDR).  Any pointer may be NULL. */
VBDR_API int vbdr_get_dims(vbdr_t h, uint32_t *R, uint32_t *w, uint32_t *words);

/* Copy the logical state to host memory (any pointer may be NULL):
 * h_dr [Z][R] uint8 (DR of LBP1 value r+1 at [j][r]), h_bs [Z] uint32
 * (gfast: bsLBP1; serial: nowLBP1; gsmall: zeros), h_reg [Z] uint8 registers
 * of the last slide. */
VBDR_API int vbdr_copy_state(vbdr_t h, uint8_t *h_dr, uint32_t *h_bs, uint8_t *h_reg,
                    void *stream);

/* Pool sums of the last slide (see vbdr_slide). */
VBDR_API int vbdr_copy_pool_sums(vbdr_t h, uint64_t *S_Z, uint64_t *V_Z, void *stream);

/* Pool sums of the last slide for VBDR_EST_LOGLOG and VBDR_EST_PCSA: L_Z =
 * sum of the Z registers, P_Z = sum of the Z PCSA statistics (0 unless
 * gsmall).  Synchronous.  Errors: VBDR_EINVAL, VBDR_ECUDA. */
VBDR_API int vbdr_copy_pool_sums_alt(vbdr_t h, uint64_t *L_Z, uint64_t *P_Z, void *stream);

/* The PCSA statistic of every physical BDR at the last slide (h_pcsa: Z
 * bytes, host).  gsmall only.  Synchronous.  Errors: VBDR_EINVAL,
 * VBDR_ECUDA. */
VBDR_API int vbdr_copy_pcsa(vbdr_t h, uint8_t *h_pcsa, void *stream);

/* Human-readable text of a vbdr_status. */
/* Bounds checks.  The library built with -DVBDR_CHECK (libvbdr_check.so,
 * next to libvbdr.so) tests every physical index, LBP1 and register value in
 * its kernels, skips an access that would leave its buffer and records it:
 * *flags receives the violations seen by this handle's kernels (bit 0: a
 * physical index >= Z, bit 1: an LBP1 > R, bit 2: a register value out of
 * range, bit 3: a planned-estimate entry out of range; always 0 in the
 * normal build) and *checked_build (may be NULL) whether the checks are
 * compiled in.  Synchronous.  Errors: VBDR_EINVAL, VBDR_ECUDA. */
VBDR_API int vbdr_check_flags(vbdr_t h, uint32_t *flags, int *checked_build);

/* Failure detection of the device-side waits.  The planned estimate waits
 * on mbarriers (its TMA ring) with a bounded wait (0.2 s): a wait that
 * expires sets the kernel's error word (vbdr_plan_status reports
 * VBDR_ETIMEOUT), the outputs concerned are NaN, and the kernel finishes, so
 * the CUDA context stays usable.  This self-test runs that wait on the GPU
 * with a limit of limit_us microseconds (1 .. 10^7) on an mbarrier that
 * nothing arrives on: it returns VBDR_ETIMEOUT once every thread of the probe
 * gave up, VBDR_OK if the wait completed (it cannot), VBDR_EINVAL for a bad
 * limit and VBDR_ECUDA on a CUDA error.  Synchronous.  Not part of the
 * paper: it only tests the library's own error path. */
VBDR_API int vbdr_selftest_bounded_wait(uint32_t limit_us, void *stream);

VBDR_API const char *vbdr_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* VBDR_H_ */
