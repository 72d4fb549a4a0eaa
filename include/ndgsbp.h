/*
 * ndgsbp.h -- C ABI of the GB300 (sm_103a) NDGSBP decoding library.
 *
 * Non-disjoint group shuffled belief propagation (NDGSBP) decoding of binary LDPC codes, after
 * Hsu, Chang, Su and Weng, "A Non-Disjoint Group Shuffled Decoding for LDPC Codes".  The
 * library builds check-node (CN) groups from a parity-check matrix H and decodes batches of
 * channel LLR frames on the GPU with a flooding, disjoint-group (GSBP) or overlapping-group
 * (NDGSBP) schedule.
 *
 * Conventions for every call:
 *   - Return value: NDGSBP_OK (0) or a negative ndgsbp_status.  On failure nothing is written
 *     to the outputs and ndgsbp_last_error() returns a message for the calling thread.  No call
 *     throws across the ABI.
 *   - Pointers named d_* are device pointers (memory on the current CUDA device), all others
 *     host pointers.  The caller owns every buffer it passes; the library owns only the opaque
 *     handles it returns and the device copies of their descriptors.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).  Device
 *     work is enqueued on it; outputs are valid once that stream has been synchronised.
 *   - Sizes are element counts unless named *_bytes.  Arrays are row-major and contiguous.
 *   - Handles are immutable after creation and may be shared by threads; one decode call at a
 *     time may use a given workspace buffer.
 */
#ifndef NDGSBP_H
#define NDGSBP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t ndgsbp_status;

#define NDGSBP_OK 0
#define NDGSBP_ERR_INVALID (-1)      /* bad argument, bad H, bad group list */
#define NDGSBP_ERR_INFEASIBLE (-2)   /* (G, r) cannot be realised on this code */
#define NDGSBP_ERR_CUDA (-3)         /* a CUDA runtime call failed (message has the detail) */
#define NDGSBP_ERR_WORKSPACE (-4)    /* workspace missing or smaller than ndgsbp_workspace_size */
#define NDGSBP_ERR_BUDGET (-5)       /* request exceeds the server's device-memory budget */
#define NDGSBP_ERR_TIMEOUT (-6)      /* a bounded device or host wait ran out */
#define NDGSBP_ERR_DEVICE (-7)       /* the kernel reported an error in its status word */
#define NDGSBP_ERR_UNSUPPORTED (-8)  /* valid request this build does not handle (e.g. degree) */
#define NDGSBP_ERR_NOMEM (-9)        /* host or device allocation failed */

/* element types */
#define NDGSBP_F32 0
#define NDGSBP_F16 1
#define NDGSBP_BF16 2
#define NDGSBP_F64 3

/* grouping units and flags for ndgsbp_groups_build */
#define NDGSBP_UNIT_CN 0         /* groups are built from single CNs */
#define NDGSBP_UNIT_LAYER 1      /* groups are built from layers of Z consecutive CNs (QC codes) */
#define NDGSBP_GROUPS_CYCLIC 1   /* G windows around a ring of units (see ndgsbp_group_sizes) */
#define NDGSBP_GROUPS_NATURAL 2  /* take units in index order instead of drawing them at random */
#define NDGSBP_GROUPS_STRUCTURED 4 /* CN units only: group 1 and the overlaps as in Step 1; the fresh
                                      CNs of group g >= 2 are picked greedily, each adding the most
                                      VNs of the previous group's VN neighbourhood not yet reached
                                      by group g (raises the CoCSG l of Sec. II-A), ties broken by
                                      the random draw order */

/* schedules */
#define NDGSBP_SCHEDULE_GROUPS 0 /* the groups of the handle: GSBP when disjoint, NDGSBP when not */
#define NDGSBP_SCHEDULE_FLOOD 1  /* one group holding every CN: standard (flooding) BP */

/* decode kernel variants */
#define NDGSBP_VARIANT_AUTO 0    /* the library's choice (ndgsbp_autotune picks by measurement) */
#define NDGSBP_VARIANT_SMEM 1    /* edge messages resident in shared memory (small codes) */
#define NDGSBP_VARIANT_GLOBAL 2  /* edge messages in per-CTA global-memory slots */
#define NDGSBP_VARIANT_QC 3      /* layered QC kernel: circulant index arithmetic, no tables */
#define NDGSBP_VARIANT_QC_GLOBAL 4 /* layered QC kernel with messages in global-memory slots */
/* values 5, 6, 8, 9 and 10 are unused (INVALID) */
#define NDGSBP_VARIANT_TILE 7      /* tile kernel: any QC window, degree <= 32, several frames per CTA */
#define NDGSBP_VARIANT_RAGGED_PER_CODE 11 /* ragged launches only: every code runs its own
                                      ndgsbp_decode plan (the library's choice for it), the launches
                                      forked onto concurrent streams and joined (same results as
                                      decoding each batch alone) */
#define NDGSBP_VARIANT_STREAM 12   /* stream kernel (QC windows too large for one thread per CN,
                                      degree <= 22): a thread per CN (or 2 lanes per CN) of a layer
                                      steps through the window's layers; messages edge-major per
                                      layer, where they live chosen by the library */
#define NDGSBP_VARIANT_STREAM_SMEM 13   /* stream kernel, all messages of a frame in shared memory */
#define NDGSBP_VARIANT_STREAM_GLOBAL 14 /* stream kernel, messages in per-CTA global-memory slots */
#define NDGSBP_VARIANT_STREAM_BULK 15   /* stream kernel, messages in per-CTA global slots with each
                                      layer's slab staged in shared memory by bulk copies (cyclic
                                      windows advancing one layer per group only) */

/* stats counters accumulated by ndgsbp_decode_ex (uint64 each) */
#define NDGSBP_STAT_FRAMES 0
#define NDGSBP_STAT_FRAME_ERRORS 1   /* decoded word != transmitted word */
#define NDGSBP_STAT_BIT_ERRORS 2     /* over the N code bits */
#define NDGSBP_STAT_UNDETECTED 3     /* syndrome satisfied but decoded word != transmitted word */
#define NDGSBP_STAT_ITERATIONS 4     /* sum of iterations used */
#define NDGSBP_STAT_UNSATISFIED 5    /* frames that stopped with a nonzero syndrome */
#define NDGSBP_STAT_INVALID 6        /* frames not decoded: a NaN or an infinity among their LLRs
                                        (counted here only, not in the counters above) */
#define NDGSBP_STATS_LEN 8

typedef struct ndgsbp_code ndgsbp_code;
typedef struct ndgsbp_groups ndgsbp_groups;
typedef struct ndgsbp_vgroups ndgsbp_vgroups;

/* Decoder parameters (Sec. II-C).  Use ndgsbp_params_default and change what you need. */
typedef struct ndgsbp_params {
    int32_t schedule;       /* NDGSBP_SCHEDULE_GROUPS or NDGSBP_SCHEDULE_FLOOD */
    int32_t max_iter;       /* I_Max >= 1 */
    int32_t msg_dtype;      /* storage type of CN->VN messages: F32, F16 or BF16 (math is FP32) */
    float llr_max;          /* clip for VN->CN inputs and CN->VN outputs of Eq. (1), in (0, 30] */
    int32_t early_stop;     /* 1: stop a frame at the first zero syndrome (Step 4 b) */
    int32_t variant;        /* NDGSBP_VARIANT_* */
    int32_t block_threads;  /* 0 = chosen by the library; else a multiple of 32, <= 1024 */
    int32_t ctas_per_sm;    /* 0 = as many as fit; else an upper bound (for the TILE variant and
                               ragged launches also the residency target that caps each CTA's
                               shared memory at 1/ctas_per_sm of the SM's) */
    int32_t frames_per_cta; /* TILE variant: frame slots per CTA, 0 = library choice, <= 16 */
    int32_t lanes_per_cn;   /* TILE variant: threads per CN (1, 2 or 4), 0 = library choice */
} ndgsbp_params;

/* Launch plan the library picked for a decode (filled by ndgsbp_decode_plan). */
typedef struct ndgsbp_plan {
    int32_t variant;        /* the NDGSBP_VARIANT_* kernel that runs (never AUTO) */
    int32_t block_threads;
    int32_t grid;           /* persistent CTAs */
    int32_t ctas_per_sm;
    int32_t max_row_degree; /* compile-time degree bound of the kernel instance */
    int32_t delta_in_smem;
    int64_t smem_bytes;     /* dynamic shared memory per CTA */
    int64_t workspace_bytes;
    int64_t stored_edges;   /* edge slots per frame including tile padding */
    int64_t edge_updates_per_iter; /* sum over groups of the CN degrees (the paper's cost unit) */
} ndgsbp_plan;

/* Optional extras of ndgsbp_decode_ex (all may be NULL / 0). */
typedef struct ndgsbp_extras {
    const uint32_t* d_ref_bits; /* transmitted word(s), packed like d_hard_bits; NULL = all-zero */
    int32_t ref_per_frame;      /* 1: d_ref_bits is [n_frames][W]; 0: one word [W] for every frame */
    uint64_t* d_stats;          /* [NDGSBP_STATS_LEN] counters, added to (caller zeroes them) */
    uint64_t* d_iter_hist;      /* [max_iter + 1] frames per iteration count, added to */
    uint64_t* d_start_ns;       /* [n_frames] device %globaltimer (ns) when each frame's decode began */
    uint64_t* d_retire_ns;      /* [n_frames] device %globaltimer (ns) when each frame retired */
    float* d_messages;          /* [n_frames][E] CN->VN messages at exit, CSR edge order */
} ndgsbp_extras;

/* Fill *p with: GROUPS schedule, max_iter 50, F32 messages, llr_max 20, early stop on, AUTO. */
void ndgsbp_params_default(ndgsbp_params* p);

/* Message for the last failed call on this thread ("" if none).  Owned by the library. */
const char* ndgsbp_last_error(void);

/* Library version string, e.g. "ndgsbp 1.0 sm_103a".  Owned by the library. */
const char* ndgsbp_version(void);

/* ---- Code (Sec. II-B: H as a bipartite graph with N VNs and M CNs) ------------------------
 * Copy an M x N parity-check matrix given in CSR form: row_ptr[M+1] (row_ptr[0] = 0,
 * nondecreasing) and col_idx[row_ptr[M]] with 0 <= col < N and no repeated column in a row.
 * lift_Z > 0 declares a QC code whose rows come in M / lift_Z layers of lift_Z CNs in which
 * every VN appears at most once (checked); 0 = unstructured.  *out receives a handle that
 * ndgsbp_code_destroy frees.  Host-only: needs no GPU.
 * Errors: INVALID for malformed CSR or a layer that repeats a VN; NOMEM. */
ndgsbp_status ndgsbp_code_create(const int32_t* row_ptr, const int32_t* col_idx, int32_t M,
                                 int32_t N, int32_t lift_Z, ndgsbp_code** out);
ndgsbp_status ndgsbp_code_destroy(ndgsbp_code* code);
/* Sizes of a code handle; any output pointer may be NULL. */
ndgsbp_status ndgsbp_code_info(const ndgsbp_code* code, int32_t* M, int32_t* N, int64_t* E,
                               int32_t* max_row_degree, int32_t* max_col_degree, int32_t* lift_Z);

/* ---- Grouping (Sec. II-A size relation, Sec. II-C Step 1) --------------------------------
 * Group sizes from G N_G - (G-1) N_G r = M over M_units units:
 *   linear:  N_G = ceil(M_units / (G - (G-1) r)), overlap o = round-half-up(r N_G); group 1 has
 *            N_G units, groups 2..G take o units from their predecessor plus fresh units that
 *            share the other M_units - N_G as evenly as possible (larger shares first).
 *   CYCLIC:  stride s = M_units / G (must divide), o = round-half-up(r s / (1 - r)), N_G = s + o;
 *            window g is units (g s + j) mod M_units of the drawn order, j < N_G.
 * Errors: INVALID when G < 1, G > M_units or r outside [0, 1); INFEASIBLE when a group would
 * get no fresh unit or the cyclic stride does not divide. */
ndgsbp_status ndgsbp_group_sizes(int32_t M_units, int32_t G, double r, int32_t flags,
                                 int32_t* NG, int32_t* overlap);

/* Step 1 of Sec. II-C.  Units (CNs, or layers of Z CNs for NDGSBP_UNIT_LAYER) are drawn with a
 * forward Fisher-Yates shuffle driven by SplitMix64(seed): draw step i swaps position i with
 * position i + (next() mod (remaining)).  G_1 takes the first N_G drawn units; G_g takes the
 * last o units of G_{g-1} followed by the next fresh units drawn (the overlap is a uniformly
 * random subset of G_{g-1} \ G_{g-2} whenever o does not exceed that set).  r = 0 gives
 * disjoint groups (GSBP); G = 1 gives one group of every CN (flooding).  The groups are kept
 * for every iteration.  Host-only.  *out receives a handle freed by ndgsbp_groups_destroy; it
 * keeps its own copy of the code.  Errors: as ndgsbp_group_sizes, INVALID for UNIT_LAYER on a
 * code without lift_Z, NOMEM. */
ndgsbp_status ndgsbp_groups_build(const ndgsbp_code* code, int32_t G, double r, uint64_t seed,
                                  int32_t unit, int32_t flags, ndgsbp_groups** out);

/* Explicit groups: grp_ptr[G+1] offsets into cn_idx[grp_ptr[G]] (0-based CN indices).  A CN
 * may appear in several groups but at most once per group.  Host-only.  Errors: INVALID. */
ndgsbp_status ndgsbp_groups_from_lists(const ndgsbp_code* code, const int32_t* grp_ptr,
                                       const int32_t* cn_idx, int32_t G, ndgsbp_groups** out);

/* Several groupings cycled by iteration -- the literal "go to Step 1" of Step 4 b), which draws
 * the groups again for every iteration: n_groupings (1..64) groupings are drawn as by
 * ndgsbp_groups_build with the seeds seed, seed + 1, ..., and iteration l of a decode uses
 * grouping (l - 1) mod n_groupings.  Decoded by the QC kernels (QC, QC_GLOBAL, TILE,
 * ragged launches, serving) when every grouping is made of whole layers with one window size;
 * the other plans return UNSUPPORTED.  ndgsbp_groups_query describes grouping 0.
 * Errors: as ndgsbp_groups_build. */
ndgsbp_status ndgsbp_groups_build_cycled(const ndgsbp_code* code, int32_t G, double r, uint64_t seed,
                                         int32_t unit, int32_t flags, int32_t n_groupings,
                                         ndgsbp_groups** out);
/* Grouping k (0 <= k < *n_groupings) of a handle, laid out as for ndgsbp_groups_query (G + 1
 * pointers, *n_entries CN indices).  Any output may be NULL.  Errors: INVALID. */
ndgsbp_status ndgsbp_groups_query_grouping(const ndgsbp_groups* groups, int32_t k, int32_t* n_groupings,
                                           int64_t* n_entries, int32_t* grp_ptr, int32_t* cn_idx);

/* Read a grouping back.  Any output may be NULL.  grp_ptr needs G+1 entries and cn_idx
 * n_entries entries (query both counts first with the arrays NULL).  cocsg is the paper's
 * l: the mean over consecutive groups of the VNs adjacent to both (Sec. I, II-B).
 * cn_updates_per_iter = sum of group sizes; edge_updates_per_iter = sum of their CN degrees. */
ndgsbp_status ndgsbp_groups_query(const ndgsbp_groups* groups, int32_t* G, int64_t* n_entries,
                                  int32_t* grp_ptr, int32_t* cn_idx, double* cocsg,
                                  int64_t* cn_updates_per_iter, int64_t* edge_updates_per_iter);
ndgsbp_status ndgsbp_groups_destroy(ndgsbp_groups* groups);

/* ---- Channel (Sec. II-C: BPSK over AWGN, L_n = 2 y_n / sigma^2) --------------------------
 * Write n_frames x N channel LLRs to d_llr (dtype F32, F16 or BF16) for the word(s) in
 * d_codeword_bits (packed like d_hard_bits; NULL = all-zero word; codeword_per_frame selects
 * [n_frames][W] or one [W]).  sigma^2 = 1 / (2 rate 10^(ebn0_db/10)).  Normals come from
 * Philox4x32-10 keyed by seed with counter (b, frame low, frame high, 0) for VNs 4b..4b+3,
 * u = ((x >> 9) + 1/2) 2^-23 (exact in FP32), and Box-Muller on (u0, u1) and (u2, u3) (cos
 * then sin).  d_llr needs the alignment of its element type (any offset into a buffer that
 * keeps it is accepted: 16-byte stores are used only where every row is 16-byte aligned).
 * Errors: INVALID (rate <= 0, bad dtype, misaligned d_llr), CUDA. */
ndgsbp_status ndgsbp_awgn_llr(const ndgsbp_code* code, int64_t n_frames, double ebn0_db,
                              double rate, uint64_t seed, const uint32_t* d_codeword_bits,
                              int32_t codeword_per_frame, void* d_llr, int32_t dtype, void* stream);

/* Raw Philox4x32-10 blocks for testing the generator: d_ctr[n][4] -> d_out[n][4] under key
 * (key0, key1).  Errors: INVALID, CUDA. */
ndgsbp_status ndgsbp_philox4x32_10(const uint32_t* d_ctr, uint32_t key0, uint32_t key1,
                                   int64_t n, uint32_t* d_out, void* stream);

/* ---- Decoding (Sec. II-C Steps 2-4) -------------------------------------------------------
 * Launch plan and workspace size for decoding n_frames frames on the current device.  Uploads
 * the grouping's device descriptor on first use on a device (allocates; call before any
 * stream capture).  Errors: INVALID, UNSUPPORTED (CN degree above 32), CUDA. */
ndgsbp_status ndgsbp_decode_plan(const ndgsbp_groups* groups, const ndgsbp_params* params,
                                 int64_t n_frames, ndgsbp_plan* plan);
ndgsbp_status ndgsbp_workspace_size(const ndgsbp_groups* groups, const ndgsbp_params* params,
                                    int64_t n_frames, size_t* bytes);

/* Decode n_frames frames of channel LLRs d_llr [n_frames][N] (llr_dtype F32, F64, F16 or
 * BF16).  Per frame and iteration l = 1..max_iter, each group g in order runs Step 2: every CN
 * of the group computes Eq. (1) from VN->CN messages L_{n->m} = P_n - L_{m->n} taken at the start
 * of the sub-iteration (P_n is the running total LLR of Eq. (3)), with inputs and outputs
 * clipped to llr_max; then P_n absorbs the change of every message of the group (Eq. (2) in
 * posterior form), in a fixed order.  After the last group, Step 4: d_n = 1 iff P_n < 0; the
 * frame stops when D H^T = 0 (early_stop) or l = max_iter.  Messages start at 0.
 * Outputs: d_hard_bits [n_frames][W], W = ceil(N/32), bit n%32 of word n/32 is d_n (required);
 * d_iters [n_frames] iterations used in 1..max_iter; d_syndrome_ok [n_frames] 1 if D H^T = 0 at
 * exit; d_posterior [n_frames][N] P_n at exit (FP32).  The last three may be NULL.
 * A frame whose channel LLRs hold a NaN or an infinity is not decoded: its hard bits and
 * posterior are 0, its iteration count 0 (outside 1..max_iter) and its syndrome flag 0 -- the
 * per-frame status word the caller reads after synchronising -- and NDGSBP_STAT_INVALID counts
 * it.  The other frames of the batch are decoded as usual.
 * d_workspace: device buffer of at least ndgsbp_workspace_size bytes, 256-byte aligned.
 * Frames are independent: a frame's result does not depend on the others in the batch.
 * Errors: INVALID, WORKSPACE, UNSUPPORTED, CUDA (launch errors; execution errors surface at
 * the caller's next synchronisation). */
ndgsbp_status ndgsbp_decode(const ndgsbp_groups* groups, const ndgsbp_params* params,
                            const void* d_llr, int32_t llr_dtype, int64_t n_frames,
                            void* d_workspace, size_t workspace_bytes, uint32_t* d_hard_bits,
                            int32_t* d_iters, uint8_t* d_syndrome_ok, float* d_posterior,
                            void* stream);

/* Status word of the last decode launched with d_workspace (read after it on `stream`, which
 * this call synchronises): 0 when every kernel completed its frames; bit 0 set when a bounded
 * wait on a bulk copy of the stream kernel (variant STREAM_BULK) gave up -- that CTA stopped and
 * the frame it held has no outputs (iteration count and flags as before the call).  Every decode
 * clears the word when it starts.  Errors: INVALID, CUDA. */
ndgsbp_status ndgsbp_workspace_status(const void* d_workspace, uint32_t* status, void* stream);

/* Test hooks for the failure path of the bounded waits (process-wide, read when a decode is
 * launched; not for production use).  skip_first_bulk_load = 1: every CTA of a STREAM_BULK
 * launch arms the mbarrier of its first bulk message load but issues no copy, so that wait can
 * only give up -- the CTA then sets bit 0 of the workspace status word and stops, leaving its
 * frame's outputs unwritten, and no copy is left in flight.  wait_polls: polls before a bounded
 * wait gives up (0 = the default, about 0.3 s).  ndgsbp_test_hooks(0, 0) restores normal
 * decoding.  Errors: INVALID. */
ndgsbp_status ndgsbp_test_hooks(int32_t skip_first_bulk_load, uint32_t wait_polls);

/* ndgsbp_decode plus the fused statistics epilogue and debug outputs of ndgsbp_extras
 * (FER/BER counters against the transmitted word, iteration histogram, retire timestamps,
 * final CN->VN messages).  extras may be NULL. */
ndgsbp_status ndgsbp_decode_ex(const ndgsbp_groups* groups, const ndgsbp_params* params,
                               const void* d_llr, int32_t llr_dtype, int64_t n_frames,
                               void* d_workspace, size_t workspace_bytes, uint32_t* d_hard_bits,
                               int32_t* d_iters, uint8_t* d_syndrome_ok, float* d_posterior,
                               const ndgsbp_extras* extras, void* stream);

/* ---- Vertical (VN-group) shuffled BP (Sec. I, the shuffled schedule over VNs it cites) ------
 * The N VNs are split into G disjoint groups, kept for every iteration.  ndgsbp_vgroups_build
 * draws them as Step 1 does for CN units with r = 0 (SplitMix64(seed) Fisher-Yates over the VNs,
 * or index order with NDGSBP_GROUPS_NATURAL, the only flag taken): G_1 takes the first
 * ceil(N / G) drawn VNs and the other groups share the rest as evenly as possible, larger
 * shares first.  ndgsbp_vgroups_from_lists takes them explicitly: grp_ptr[G+1] (grp_ptr[0] = 0,
 * grp_ptr[G] = N, no empty group) into grp_vn[N], which lists every VN exactly once.  Host-only;
 * *out is freed by ndgsbp_vgroups_destroy and keeps its own reference to the code.
 * Errors: INVALID (bad lists, unknown flag, G < 1 or G > N), INFEASIBLE (as ndgsbp_group_sizes),
 * NOMEM. */
ndgsbp_status ndgsbp_vgroups_build(const ndgsbp_code* code, int32_t G, uint64_t seed, int32_t flags,
                                   ndgsbp_vgroups** out);
ndgsbp_status ndgsbp_vgroups_from_lists(const ndgsbp_code* code, const int32_t* grp_ptr, const int32_t* grp_vn,
                                        int32_t G, ndgsbp_vgroups** out);
/* Read the groups back (any output may be NULL): G, grp_ptr[G+1], grp_vn[N], and the largest
 * number of edges of one group's VNs. */
ndgsbp_status ndgsbp_vgroups_query(const ndgsbp_vgroups* vgroups, int32_t* G, int32_t* grp_ptr, int32_t* grp_vn,
                                   int32_t* max_group_edges);
ndgsbp_status ndgsbp_vgroups_destroy(ndgsbp_vgroups* vgroups);

/* Workspace bytes of ndgsbp_decode_vertical for n_frames frames on the current device (the
 * CN->VN messages of a frame stay in shared memory when 8 N bytes plus the messages fit in
 * one CTA's, else they use a workspace slot per CTA; variant SMEM requires the former, GLOBAL
 * takes the latter, AUTO chooses).  Of params only max_iter, msg_dtype, llr_max, early_stop,
 * variant (AUTO, SMEM or GLOBAL), block_threads (0 or a multiple of 32 up to 512) and
 * ctas_per_sm are used.  Errors: INVALID, UNSUPPORTED (8 N bytes above a CTA's shared memory,
 * or SMEM when the messages do not fit), CUDA. */
ndgsbp_status ndgsbp_vertical_workspace_size(const ndgsbp_vgroups* vgroups, const ndgsbp_params* params,
                                             int64_t n_frames, size_t* bytes);

/* Decode with the vertical schedule.  Per frame and iteration l = 1..max_iter, for each VN group
 * in order: every edge (m, n) with n in the group gets L_{m->n} by Eq. (1) from the VN->CN
 * messages L_{n'->m} of the CN's other edges as they stand when the group starts (inputs and
 * output clipped to llr_max); then every edge of the group's VNs gets L_{n->m} = L_n + the sum
 * of L_{m'->n} over the VN's other CNs (Eq. (2); the kernel holds it as P_n - L_{m->n} with
 * P_n = L_n + the sum over all of the VN's CNs).  After the last group, Step 4 of Sec. II-C:
 * d_n = 1 iff P_n < 0, stop when D H^T = 0 (early_stop) or l = max_iter.  Messages start at 0,
 * VN->CN messages at L_n.  G = 1 is flooding.  Inputs, outputs, extras (statistics, histogram,
 * timestamps, final CN->VN messages in CSR order), NaN/infinity handling, frame independence
 * and workspace rules as ndgsbp_decode_ex.  Uploads the groups' tables on first use on a device
 * (allocates).  Errors: INVALID, WORKSPACE, UNSUPPORTED, CUDA. */
ndgsbp_status ndgsbp_decode_vertical(const ndgsbp_vgroups* vgroups, const ndgsbp_params* params,
                                     const void* d_llr, int32_t llr_dtype, int64_t n_frames,
                                     void* d_workspace, size_t workspace_bytes, uint32_t* d_hard_bits,
                                     int32_t* d_iters, uint8_t* d_syndrome_ok, float* d_posterior,
                                     const ndgsbp_extras* extras, void* stream);

/* ---- Ragged batches: several codes in one persistent launch --------------------------------
 * One code's part of a ragged batch: its grouping (a QC code grouped in whole layers), its
 * channel LLRs [n_frames][N] and its outputs, laid out as for ndgsbp_decode.  d_stats,
 * d_start_ns and d_retire_ns are optional (see ndgsbp_extras). */
typedef struct ndgsbp_batch {
    const ndgsbp_groups* groups;
    const void* d_llr;
    int32_t llr_dtype;
    int64_t n_frames;
    uint32_t* d_hard_bits;
    int32_t* d_iters;
    uint8_t* d_syndrome_ok;
    float* d_posterior;
    uint64_t* d_stats;
    uint64_t* d_start_ns;
    uint64_t* d_retire_ns;
    int32_t frames_per_cta;  /* 0 = library choice */
    int32_t lanes_per_cn;    /* 0 = library choice */
} ndgsbp_batch;

typedef struct ndgsbp_ragged ndgsbp_ragged;

/* Plan one persistent tile-kernel launch over n_batches <= 8 batches of different codes: each
 * code keeps its own schedule (Sec. II-C Steps 2-4 with its groups) and per-frame early stop;
 * CTAs take tiles of frames of any code from one list (largest codes first) and refill frame
 * slots as frames retire.  params gives max_iter, msg_dtype, llr_max, early_stop, block_threads
 * (shared by every code) and ctas_per_sm, the residency target k: every CTA's shared memory is
 * capped at 1/k of the SM's, and a code whose messages do not fit under the cap keeps them in
 * global memory (0 = 2 CTAs per SM when every code fits, else 1).  With params->variant =
 * NDGSBP_VARIANT_RAGGED_PER_CODE the handle instead keeps one ndgsbp_decode plan per code (the
 * library's default choice, e.g. the layered QC kernel where it applies; block_threads,
 * ctas_per_sm and the batches' tile shapes are then ignored) and a launch forks them onto
 * concurrent streams that the caller's stream joins; a graph replay holds all of them.  Any
 * grouping is accepted in that mode.  The batches' buffers are recorded in the handle: later
 * launches reuse them, so refill their contents rather than moving them.  Allocates the tile
 * list and the launch's workspace (owned by the handle; call before any stream capture).
 * Errors: INVALID, UNSUPPORTED (a code that is not QC in whole layers, degree > 32), CUDA, NOMEM. */
ndgsbp_status ndgsbp_ragged_create(const ndgsbp_batch* batches, int32_t n_batches,
                                   const ndgsbp_params* params, ndgsbp_ragged** out);
/* Launch plan (variant TILE; grid, block, shared bytes) and number of tiles; in the per-code
 * mode variant RAGGED_PER_CODE, the summed grids, the largest block and shared size, and the
 * number of codes in n_tiles. */
ndgsbp_status ndgsbp_ragged_info(const ndgsbp_ragged* ragged, ndgsbp_plan* plan, int32_t* n_tiles);
/* Enqueue the launch on stream: a counter reset and one kernel (per-code mode: a fork onto the
 * handle's streams, one reset and kernel per code, and a join back into stream). */
ndgsbp_status ndgsbp_ragged_launch(ndgsbp_ragged* ragged, void* stream);
/* The same launch through a CUDA graph: the first call on a stream captures the reset and the
 * kernel into a graph and instantiates it, later calls replay it (one cudaGraphLaunch). */
ndgsbp_status ndgsbp_ragged_graph_launch(ndgsbp_ragged* ragged, void* stream);
ndgsbp_status ndgsbp_ragged_destroy(ndgsbp_ragged* ragged);

/* ---- Autotuning (the paper has no counterpart) ---------------------------------------------
 * ndgsbp_autotune times candidate launch shapes of ndgsbp_decode on the caller's frames d_llr
 * [n_frames][N] (a representative sample: the iteration counts follow its noise level) and
 * returns the fastest in result->best: params with variant, block_threads, ctas_per_sm,
 * frames_per_cta and lanes_per_cn filled in (the other fields as given).  Candidates are the
 * library's default choice, the QC kernel at 0/1/2 CTAs per SM (messages in shared memory) and
 * at 0/2/3/4 CTAs per SM (messages in global memory), the stream kernel's three storage modes at
 * 1 and 2 lanes per CN, and tile shapes (1, 2 or 4 lanes per CN x
 * 1..16 frames per CTA x 128..512 threads, at the default residency and at 1 CTA per SM) that
 * the plan accepts.  Each
 * candidate is an ordinary decode into the tuner's own scratch buffers: one untimed call, then
 * the median of three timed by CUDA events on a private stream.  Shapes with the same lanes
 * per CN give bit-identical results; more lanes per CN split a CN's edges between lanes and so
 * change the order of FP32 additions in Eq. (1), i.e. results agree to rounding.
 * Results are cached in memory under a content key (the code, its groups, schedule, max_iter,
 * msg_dtype, early_stop, llr_max, block_threads, llr_dtype, log2 of n_frames, device name and
 * SM count) and, with cache_path non-NULL, appended to that text file (loaded on first use) so
 * later processes skip the timing.  flags: NDGSBP_TUNE_TILE_ONLY restricts the candidates to
 * the TILE variant and, when params->block_threads is set, keeps that block size.
 * Allocates and frees device memory (not during stream capture).
 * Errors: INVALID, UNSUPPORTED (no shape fits), NOMEM, CUDA. */
#define NDGSBP_TUNE_TILE_ONLY 1

typedef struct ndgsbp_tune_result {
    ndgsbp_params best;
    double best_ms;         /* median decode time of the sample with best */
    double default_ms;      /* the same for the library's default choice (0 with TILE_ONLY) */
    int32_t candidates;     /* shapes timed */
    int32_t from_cache;     /* 1 when the result came from the cache (nothing was timed) */
} ndgsbp_tune_result;

ndgsbp_status ndgsbp_autotune(const ndgsbp_groups* groups, const ndgsbp_params* params,
                              const void* d_llr, int32_t llr_dtype, int64_t n_frames, int32_t flags,
                              const char* cache_path, ndgsbp_tune_result* result);

/* Tile shape of a ragged launch: for each block size 128, 256, 384, 512 the per-code tile shape
 * (frames_per_cta, lanes_per_cn) is tuned with ndgsbp_autotune (TILE_ONLY) on the first
 * sample_frames frames of each batch (all when <= 0); then the whole ragged launch over the
 * batches is timed (one untimed launch, best of two timed) at 1, 2, 3 and 4 CTAs per SM, with
 * frame slots capped to fit, and the per-code mode (NDGSBP_VARIANT_RAGGED_PER_CODE) is timed
 * the same way; the fastest (block size, residency) or the per-code mode wins.  On return
 * batches[i].frames_per_cta / lanes_per_cn and *params_out (variant TILE with block_threads and
 * ctas_per_sm, or RAGGED_PER_CODE) hold the winner, and *best_ms its launch time.  The timing launches write the batches'
 * output buffers.  Errors: as ndgsbp_autotune and ndgsbp_ragged_create. */
ndgsbp_status ndgsbp_ragged_autotune(ndgsbp_batch* batches, int32_t n_batches,
                                     const ndgsbp_params* params, int64_t sample_frames,
                                     const char* cache_path, ndgsbp_params* params_out,
                                     double* best_ms);

/* ---- Serving: continuous batching of decode requests ---------------------------------------
 * A server owns, per code, a pool of frame slots (posterior and messages of running frames in
 * device memory; LLR staging and outputs in pinned host memory that the kernel reads and writes
 * directly) sized so that all pools fit hbm_budget_bytes (split in proportion to weights; NULL =
 * equal shares).  Staging threads of the library place the frames of queued
 * requests into free slots in arrival order (copying their LLRs while epochs run); a worker
 * thread runs epochs in which every running frame advances by at most epoch_iters iterations
 * (its state stays in device memory between epochs), and retires frames whose syndrome is zero
 * (Step 4 b) or that reached params->max_iter; the worker copies an epoch's retired frames out
 * and frees their slots while the next epoch runs on the GPU.
 * A request completes when all its frames have retired.  An epoch is one serving launch per
 * pool whose plain decode (variant AUTO) would use the layered QC kernel or the stream kernel,
 * of that kernel (forked onto the pool's own stream; a stream pool keeps its messages in shared
 * or global memory, never bulk-staged), and one serving launch of the tile kernel over the
 * other pools; with params->variant = NDGSBP_VARIANT_TILE every pool runs on the tile kernel.
 * Every frame is decoded exactly as by ndgsbp_decode with the kernel of its pool (variant AUTO
 * for a pool on the QC or stream kernel, TILE for the others), whatever else is in flight.
 * Errors: INVALID, BUDGET (a pool would get no slot), UNSUPPORTED (a code that is not QC in
 * whole layers, or that the tile kernel does not take), CUDA, NOMEM. */
typedef struct ndgsbp_server ndgsbp_server;

typedef struct ndgsbp_server_stats {
    int64_t requests_submitted, requests_completed;
    int64_t frames_completed, frame_errors_unsatisfied;
    int64_t epochs;
    int64_t iterations;          /* frame-iterations run */
    double busy_seconds;         /* host time with at least one frame on the device */
    int64_t slots_total, slots_in_use;
    double admit_seconds;        /* staging threads' time copying admitted frames' LLRs, summed (overlaps epochs) */
    double device_seconds;       /* worker time waiting for epochs to finish (after the overlapped harvest) */
    double harvest_seconds;      /* worker time copying retired frames' outputs (overlaps the next epoch) */
    int64_t launches;            /* kernels launched by the epochs (admit, QC, stream and tile launches) */
} ndgsbp_server_stats;

ndgsbp_status ndgsbp_server_create(const ndgsbp_groups* const* codes, int32_t n_codes,
                                   const double* weights, const ndgsbp_params* params,
                                   size_t hbm_budget_bytes, int32_t epoch_iters,
                                   ndgsbp_server** out);
/* Queue a request of n_frames frames of code `code` (index into the create-time list):
 * host_llr [n_frames][N] FP32 is read during admission and must stay valid until the request
 * completes; the outputs (laid out as for ndgsbp_decode, host memory, host_iters and
 * host_syndrome_ok may be NULL) are written before completion is reported.  *ticket identifies
 * the request.  Thread-safe. */
ndgsbp_status ndgsbp_server_submit(ndgsbp_server* server, int32_t code, const float* host_llr,
                                   int64_t n_frames, uint32_t* host_hard_bits, int32_t* host_iters,
                                   uint8_t* host_syndrome_ok, int64_t* ticket);
/* *done = 1 once the request completed; *latency_ms = completion - submission (host clock).
 * Completion is reported once: after poll reported done (or wait returned OK) the ticket is
 * released and later calls with it return INVALID. */
ndgsbp_status ndgsbp_server_poll(ndgsbp_server* server, int64_t ticket, int32_t* done,
                                 double* latency_ms);
/* Block until the request completes or timeout_ms passes (TIMEOUT). */
ndgsbp_status ndgsbp_server_wait(ndgsbp_server* server, int64_t ticket, int32_t timeout_ms,
                                 double* latency_ms);
ndgsbp_status ndgsbp_server_stats_get(ndgsbp_server* server, ndgsbp_server_stats* stats);
/* Stops the worker (finishing the epoch in flight) and frees the pools. */
ndgsbp_status ndgsbp_server_destroy(ndgsbp_server* server);

/* ---- Gaussian-approximation analysis (Sec. III), FP64 on the GPU ----------------------------
 * The GA mean recursion for the flooding schedule (Eq. (4) with every other CN of class a, then
 * Eqs. (15)-(16)): mu_v,i = mu0 + (i - 1) mu_c and mu_c <- sum_j rho_j Phi^-1(1 - (1 - sum_i
 * lambda_i Phi(mu_v,i))^(j-1)), from mu_c = 0, with mu0 = 2 / sigma^2 and sigma^2 =
 * 1 / (2 rate 10^(Eb/N0 / 10)), evaluated for n_points Eb/N0 values at once in FP64 (one warp per
 * point).  phi_kind: EXACT = Eq. (14) by the trapezoidal rule (769 nodes over x in [-12, 12], T =
 * mu + 2 sqrt(mu) x), CLOSED = the closed-form approximation of the GA analysis the paper cites
 * (the form that reproduces Table I's thresholds).  lambda[i] / rho[j]: edge-perspective degree
 * fractions indexed by degree, i <= dv_max <= 64, j <= dc_max <= 64 (Sec. II-B).  Per point (host
 * arrays, written before return): converged = 1 when mu_c reached mu_cap (error-free decoding),
 * iters = the iteration at which it did, or at which mu_c stopped moving (a fixed point: relative
 * change <= 1e-12), or max_iter; mu_c = the last CN mean.  Synchronous; allocates device memory.
 * Errors: INVALID, CUDA. */
#define NDGSBP_GA_PHI_EXACT 0
#define NDGSBP_GA_PHI_CLOSED 1
ndgsbp_status ndgsbp_ga_flood(const double* lambda, int32_t dv_max, const double* rho, int32_t dc_max,
                              double rate, const double* ebn0_db, int32_t n_points, int32_t phi_kind,
                              int32_t max_iter, double mu_cap, uint8_t* converged, int32_t* iters,
                              double* mu_c);
/* GA threshold: the smallest Eb/N0 in [lo_db, hi_db] at which ndgsbp_ga_flood converges, found
 * by refining the bracketing pair of a grid of at most 64 points (no finer than tol_db where that
 * takes fewer) until it is narrower than tol_db; the upper end of the final pair is returned.  Errors: INVALID, INFEASIBLE (no convergence at hi_db), CUDA. */
ndgsbp_status ndgsbp_ga_flood_threshold(const double* lambda, int32_t dv_max, const double* rho,
                                        int32_t dc_max, double rate, int32_t phi_kind,
                                        int32_t max_iter, double mu_cap, double lo_db, double hi_db,
                                        double tol_db, double* threshold_db);

/* The GA recursion for the group schedules of Sec. III: G groups (1..64) with overlap ratio r in
 * [0, 1) (r = 0: disjoint groups, GSBP).  Per iteration and group g = 1..G the mean of a VN's
 * other CN messages mixes class a (not updated yet in this iteration, mean mu_c of the previous
 * iteration), class b (the overlap with group g - 1, fraction z = r / D of Eq. (12)) and class d
 * (updated, fraction x = 1 / D for g = 1 (Eq. (10)) and y = g (1 - r) / D otherwise (Eq. (11)),
 * with mean from Eqs. (6)-(7)), D = G - (G - 1) r; Eq. (8) with the weights of Eq. (9) is then
 * mu0 + (i - 1)(y mu_d + z mu_b + (1 - y - z) mu_a) since it is linear in (p, q).  The group's
 * class-c CN output follows Eqs. (15)-(16); a class-b CN (g >= 2, r > 0) uses the weights of
 * Eq. (9) restricted to p >= 1 (at least one updated neighbour).  Eq. (17) gives the iteration's
 * mean.  Readings of points the paper leaves open: the current group's own term in Eqs. (6)-(7)
 * is its output of the previous iteration (what its fresh CNs hold during the sub-iteration), and
 * for g = 1 class d is group 1's previous output.  Inputs, outputs and stop rule as
 * ndgsbp_ga_flood.  Synchronous; allocates device memory.  Errors: INVALID, CUDA. */
ndgsbp_status ndgsbp_ga_groups(const double* lambda, int32_t dv_max, const double* rho, int32_t dc_max, double rate,
                               int32_t G, double r, const double* ebn0_db, int32_t n_points, int32_t phi_kind,
                               int32_t max_iter, double mu_cap, uint8_t* converged, int32_t* iters, double* mu_c);
/* GA threshold of the group schedule, found as by ndgsbp_ga_flood_threshold.
 * Errors: INVALID, INFEASIBLE, CUDA. */
ndgsbp_status ndgsbp_ga_groups_threshold(const double* lambda, int32_t dv_max, const double* rho, int32_t dc_max,
                                         double rate, int32_t G, double r, int32_t phi_kind, int32_t max_iter,
                                         double mu_cap, double lo_db, double hi_db, double tol_db,
                                         double* threshold_db);

/* ---- Measurement aid (the paper has no counterpart) ----------------------------------------
 * Launch `blocks` x `threads` threads that each run iters x 8 independent FP32 MUFU operations of
 * kind op (0: ex2.approx, 1: rcp.approx, 2: lg2.approx -- the three of each edge-update of Eq. (1))
 * on `stream`, for timing the XU pipe's rate with events around the launch.  d_sink: a device
 * buffer of `blocks` floats (never written in practice).  Errors: INVALID, CUDA. */
ndgsbp_status ndgsbp_mufu_probe(int32_t op, int64_t iters, int32_t blocks, int32_t threads, float* d_sink,
                                void* stream);

/* ---- Decoding without allocating (the paper has no counterpart) ---------------------------
 * ndgsbp_decode_static is ndgsbp_decode without a workspace: it allocates no device memory.  It
 * is for callers that cannot allocate while they decode -- a real-time receive loop that may
 * not call cudaMalloc (the call can synchronise the device and its latency is unbounded), or a
 * process whose device memory is already handed out by another allocator, so that a new
 * allocation would fail.  The kernels' scratch (the frame counter, and the per-CTA message slots
 * of the global-memory variants) lives in one static device array of
 * NDGSBP_STATIC_SCRATCH_BYTES bytes inside this library, which every GPU that loads the library
 * holds until the process exits.
 *   - The first call on a device looks up the array's device address (a one-time set-up per
 *     device); make that first call before any stream capture.  The library keeps that address,
 *     like the grouping tables it uploads, for the life of the process: after a device reset
 *     (cudaDeviceReset) neither is valid, so do not reset a device while this library uses it.
 *   - The grouping's tables must already be on the device: call ndgsbp_decode_plan with the same
 *     parameters, on that device, during set-up (that call uploads them).  Otherwise INVALID.
 *   - A launch that needs more scratch than the array holds is rejected with WORKSPACE (lower
 *     ctas_per_sm, keep messages in shared memory, or use ndgsbp_decode with a workspace).
 *   - Every call shares the one array and clears its counter on `stream`; calls whose work
 *     overlaps on the GPU (other streams, other threads) race on it and corrupt each other's
 *     results, so issue them one after another on one stream.
 * Arguments, outputs and the remaining errors are those of ndgsbp_decode. */
#define NDGSBP_STATIC_SCRATCH_BYTES (16u * 1024u * 1024u)
ndgsbp_status ndgsbp_decode_static(const ndgsbp_groups* groups, const ndgsbp_params* params,
                                   const void* d_llr, int32_t llr_dtype, int64_t n_frames,
                                   uint32_t* d_hard_bits, int32_t* d_iters, uint8_t* d_syndrome_ok,
                                   float* d_posterior, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* NDGSBP_H */
