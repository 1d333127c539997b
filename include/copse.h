/*
 * copse.h -- C ABI of the GB300 (sm_103a) COPSE secure decision-forest library.
 *
 * COPSE (Malik et al., "Vectorized Secure Evaluation of Decision Forests",
 * PLDI'21) compiles a plaintext decision forest into vectorised structures
 * (Section 4.2) and evaluates Algorithm 1 (Section 4.3) over packed BGV
 * ciphertexts: SecComp of the replicated feature vector against the padded
 * threshold vector, a reshuffle matrix-vector product, one product plus mask
 * per level, and the product across levels.  The runtime interface follows
 * Section 5 ("COPSE Runtime": encrypt models and feature vectors, run secure
 * inference) and the workflow of Section 3.2.
 *
 * Conventions for every call:
 *   - Status: 0 on success, a negative COPSE_E* code on failure; nothing
 *     aborts.  copse_last_error() gives a message for the calling thread.
 *   - Ownership: the library allocates and frees every handle; inputs are
 *     copied or only read during the call; outputs go to caller-owned buffers
 *     or to new handles the caller destroys with the matching *_destroy.
 *   - Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy
 *     default stream).  Calls that take host output buffers synchronise the
 *     stream before returning; calls marked "async" only enqueue work.
 *   - Device: handles are bound to the device of the context that made them;
 *     the caller keeps that device current.
 *   - Threads: one context per host thread; handles are not internally locked.
 *
 * Plaintext modulus: t = 65537 (prime, = 1 mod 2^17), N slots in two rows of
 * N/2.  Slot values are bits; AND is a product, XOR a + b - 2ab.  The paper's
 * BGV runs at plaintext modulus 2 in HElib; with a power-of-two ring degree
 * that modulus gives a single slot, so t = 65537 carries the same bit circuit.
 */
#ifndef COPSE_H
#define COPSE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int copse_status;
#define COPSE_OK 0
#define COPSE_EINVAL (-1)   /* bad argument, size or shape                      */
#define COPSE_ENOMEM (-2)   /* device or host allocation failed                 */
#define COPSE_EPARSE (-3)   /* malformed forest text                            */
#define COPSE_ECUDA (-4)    /* a CUDA runtime call failed                       */
#define COPSE_ENOKEY (-5)   /* a rotation key the model needs is missing        */
#define COPSE_ELEVEL (-6)   /* the prime chain is too short for the circuit    */
#define COPSE_EFIT (-7)     /* the model's slot block does not fit a slot row   */
#define COPSE_EADMIT (-8)   /* admission refused: device memory or a full queue */
#define COPSE_ETIMEOUT (-9) /* a wait ran out before the result was ready      */

/* Ring and RNS parameters.  All primes are = 1 mod 2*N*t and below
 * 2^prime_bits, chosen in decreasing order: n_primes ciphertext primes, then
 * alpha = ceil(n_primes / dnum) special primes for hybrid key switching. */
typedef struct copse_params {
    uint32_t log_n;      /* ring degree N = 2^log_n, 4 <= log_n <= 15 (2N | t-1)  */
    uint32_t prime_bits; /* bit length of every prime, 36 <= prime_bits <= 55     */
    uint32_t n_primes;   /* ciphertext primes L, 1 <= L <= 40                      */
    uint32_t dnum;       /* key-switching digits, 1 <= dnum <= L                   */
} copse_params;

typedef struct copse_ctx copse_ctx;     /* device, prime tables, NTT tables            */
typedef struct copse_model copse_model; /* compiled forest (host) + its device plaintexts */
typedef struct copse_keys copse_keys;   /* secret and public key (the data owner's)   */
typedef struct copse_evk copse_evk;     /* relinearisation and rotation keys (server) */
typedef struct copse_ctbuf copse_ctbuf; /* an ordered set of device ciphertexts        */

typedef struct copse_model_info {
    uint32_t n_features;  /* features of a query                                   */
    uint32_t precision;   /* p: bits of every feature and threshold (Section 4.1.2) */
    uint32_t K;           /* maximum multiplicity (Section 4.1.1)                    */
    uint32_t q;           /* quantised branching K * n_features                      */
    uint32_t b;           /* branching: number of branch nodes                       */
    uint32_t n_leaves;    /* L: slots of the result, one per leaf                    */
    uint32_t depth;       /* d: number of levels                                     */
    uint32_t n_trees;
    uint32_t n_classes;   /* label names on the first line of the model text        */
    uint32_t block;       /* slots per query block (power of two >= L+b+q-2)          */
    uint32_t n_rot_reshuffle; /* nonzero rotation amounts of the reshuffle product   */
    uint32_t n_rot_level;     /* nonzero rotation amounts shared by the level products */
    uint32_t levels_used; /* primes the circuit drops: 3 + ceil(log2 p) + ceil(log2 d) (+1 shuffled) */
    uint32_t n_out;       /* result slots per query: n_leaves, or the shuffled and padded length */
    uint32_t n_segments;  /* row segments: 1, or the number of slot blocks one query spans when the
                             forest is split into contiguous groups of trees (copse_compile_forest) */
    uint32_t block_branches; /* branches and leaves one slot block is laid out for: b and */
    uint32_t block_leaves;   /* n_leaves, or the largest segment's (level matrices: d of L x b) */
} copse_model_info;

/* Message for the last failed call on this thread (never NULL). */
const char *copse_last_error(void);

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device`: selects the primes, builds the
 * NTT and base-conversion tables on the device.  EINVAL on out-of-range
 * parameters, ECUDA/ENOMEM on device failure. */
copse_status copse_ctx_create(const copse_params *params, int device, copse_ctx **out);
void copse_ctx_destroy(copse_ctx *ctx);

/* Device status of the context: bits that kernels with bounded waits set when a
 * wait ran out (COPSE_DEV_*), read after the device finished all queued work and
 * then cleared.  COPSE_OK with *status = 0 when nothing ran out; COPSE_ETIMEOUT
 * with the bits in *status otherwise (the results of the affected calls are
 * not valid).  A wait of the encrypted-model multiply-accumulate (the tensor-core
 * kernel of copse_infer on an encrypted model) gives up after 2 s. */
#define COPSE_DEV_MAC_WAIT 1 /* the encrypted-model multiply-accumulate */
copse_status copse_ctx_device_status(copse_ctx *ctx, int *status);

/* The n_primes + alpha primes (ciphertext primes first) into out[0..cap). */
copse_status copse_ctx_primes(const copse_ctx *ctx, uint64_t *out, size_t cap, size_t *count);

/* ---------------------------------------------------------------- models */

/* Compile a forest (Section 5, "Input Representation"): the first line lists
 * the label (class) names; each further line is one tree in preorder, a branch
 * written "b <feature> <threshold>" followed by its left then right subtree, a
 * leaf "l <class>".  A branch sends x[feature] < threshold to the right
 * (true) child.  Builds the padded threshold vector, the reshuffling matrix,
 * the level matrices and masks (Section 4.2) for rings of degree 2^log_n.
 * Host only; touches no device.  n_features = 0 takes the largest feature
 * index + 1.  EPARSE on malformed text, EINVAL on a threshold >= 2^precision,
 * a feature >= n_features or a class index out of range.
 * Row segments: when one query block (a power of two >= L + b + q - 2 slots)
 * would exceed a slot row (N/2), the trees are split into the smallest power of
 * two S of contiguous groups (tree t in group floor(S * branches before t /
 * all branches)) that are compiled alike with a common K and depth, such that
 * the common block fits a row; query j then owns blocks j S .. j S + S - 1
 * (block s: group s), N / (S block) queries per ciphertext, and its result bits
 * are the groups' leaves in order.  EFIT if no such split exists. */
copse_status copse_compile_forest(const char *text, size_t len, uint32_t precision, uint32_t n_features,
                                  uint32_t log_n, copse_model **out);
void copse_model_destroy(copse_model *model);
copse_status copse_model_info_get(const copse_model *model, copse_model_info *info);

/* Compiled structures, for inspection and host-side parity tests.
 *   thr_slot[q], slot_branch[q]: padded threshold vector and the branch each
 *     padded slot holds (-1 = sentinel, Section 4.2.1);
 *   R[b*q]: reshuffling matrix, row-major (Section 4.2.2);
 *   lvl[d*L*b]: level matrices k = 1..d, row-major (Section 4.2.3);
 *   mask[d*L]: level masks (Section 4.2.4);
 *   br_level[b]: level of each branch (Section 4.1.1).
 * Any pointer may be NULL to skip that array. */
copse_status copse_model_export(const copse_model *model, uint32_t *thr_slot, int32_t *slot_branch, uint8_t *R,
                                uint8_t *lvl, uint8_t *mask, uint32_t *br_level);

/* Nonzero rotation amounts: reshuffle then level products, ascending in each
 * (baby and giant steps when a baby-step size is set). */
copse_status copse_model_rotations(const copse_model *model, uint32_t *reshuffle, uint32_t *level);

/* Baby-step / giant-step matrix products (the diagonal method of Section 4.1.2
 * in Halevi and Shoup's BSGS form): diagonal i = k g + j is multiplied, shifted
 * by k g inside the query block, with rot(v, j); the sums per giant step k g are
 * rotated by k g and added, with one ModDown for all giant steps of a matrix.
 * g_reshuffle, g_level: baby-step sizes for the reshuffle and for the level
 * products; 0 keeps the plain method (one rotation per nonzero diagonal).
 * About 2 sqrt(width) rotation keys instead of one per diagonal.  Set before
 * copse_keygen (the key set follows the setting); drops the model's device
 * copy if the setting changes.  EINVAL if a shifted diagonal would leave the
 * query block. */
copse_status copse_model_set_bsgs(copse_model *model, uint32_t g_reshuffle, uint32_t g_level);
copse_status copse_model_get_bsgs(const copse_model *model, uint32_t *g_reshuffle, uint32_t *g_level);

/* Fused level matrices: Algorithm 1 multiplies Decisions by the reshuffling
 * matrix R (Section 4.2.2), then Branches by each level matrix (Section 4.2.3).
 * With on != 0 the two products are folded into one per level: F_k = S_k R
 * with S_k = (1 - 2 Mask_k) Lvl_k the signed level matrix (XOR folded in), an
 * L x q matrix with one entry per row, applied to Decisions by the diagonal
 * method; the rotations of Decisions serve every level.  No Branches vector,
 * no reshuffle key switches, one prime fewer (levels_used); the decrypted leaf
 * bits are the same.  The baby-step size of copse_model_set_bsgs' g_reshuffle
 * applies to these q-wide products (g_level is unused).  Plaintext model only
 * (EINVAL with an encrypted-mode model).  Set before copse_keygen; drops the
 * model's device copy when it changes. */
copse_status copse_model_set_fused(copse_model *model, int on);
int copse_model_is_fused(const copse_model *model);  /* 1 when fused, else 0 */

/* Encrypted-model mode (Section 3.1's model owner Maurice is the data owner
 * Diane, Section 8.3): the threshold planes, every diagonal of the reshuffle
 * and level matrices, zero ones included, and the level masks are encrypted,
 * p + q + d(b+1) ciphertexts (Table 1d), and the products of Algorithm 1
 * become ciphertext x ciphertext (relinearised once per baby-step sum).
 * copse_model_set_encrypted selects the mode before copse_keygen (the mode
 * needs a rotation for every diagonal: use a baby-step plan for large models).
 * copse_encrypt_model then encrypts the model under `keys`' secret key on ctx:
 * secret-key encryptions at the levels of use whose masks c1 are drawn from
 * `seed` in evaluation form, so only c0 is stored on the device (words:
 * p L + q lvl_D + d (b+1) lvl_B times N) and c1 is regenerated where the
 * products consume it.  copse_infer on the model then runs the encrypted
 * circuit; EINVAL if the model has no encryption for that context or was
 * encrypted for another baby-step plan.  Changing the mode or the plan drops
 * the encryption. */
copse_status copse_model_set_encrypted(copse_model *model, int on);
int copse_model_is_encrypted(const copse_model *model);  /* 1 in encrypted-model mode, else 0 */
copse_status copse_encrypt_model(copse_ctx *ctx, const copse_keys *keys, copse_model *model, uint64_t seed);

/* Label shuffle with padding (Section 7.2, "Returning classification
 * bitvectors"; the paper describes it and leaves it unimplemented): the server
 * permutes the result bitvector by one more plaintext matrix product (diagonal
 * method over signed shifts) and hands out the codebook permuted alike, padded
 * with extra labels whose bits are always 0.  src[j] = the leaf output slot j
 * carries (-1 = padding), codebook[j] = its class; every leaf exactly once,
 * n_leaves <= n_out <= block; n_out = 0 turns the shuffle off.  Costs one more
 * prime (levels_used + 1) and one rotation key per distinct shift; results,
 * copse_decrypt_labels and sessions then give n_out bits per query (info.n_out).
 * Host only; set before copse_keygen.  EINVAL on a malformed plan. */
copse_status copse_model_set_shuffle(copse_model *model, const int32_t *src, size_t n_out, const uint32_t *codebook);
/* The class of each result slot, classes[0..n_out): the codebook (leaf classes
 * in preorder when not shuffled). */
copse_status copse_model_codebook(const copse_model *model, uint32_t *classes);

/* Model ciphertext `index` (threshold planes, reshuffle diagonals, level
 * diagonals level by level, masks) in coefficient form [2][level][N] into
 * out[0..words), host memory, c1 regenerated.  For parity tests. */
copse_status copse_encmodel_export(copse_ctx *ctx, const copse_model *model, size_t index, uint64_t *out,
                                   size_t words);

/* Plaintext classification (Section 2.1): one bit per leaf per query,
 * out_bits[n_queries * n_leaves]; feats[n_queries * n_features] on the host. */
copse_status copse_classify_plain(const copse_model *model, const uint32_t *feats, size_t n_queries,
                                  uint8_t *out_bits);

/* ---------------------------------------------------------------- keys */

/* Generate the secret key, public key, relinearisation key and one rotation
 * key for every rotation amount any of `models` uses, from the counter-based
 * generator seeded with `seed`.  All keys stay in device memory.  Synchronous. */
copse_status copse_keygen(copse_ctx *ctx, uint64_t seed, const copse_model *const *models, size_t n_models,
                          copse_keys **keys, copse_evk **evk);
void copse_keys_destroy(copse_keys *keys);
void copse_evk_destroy(copse_evk *evk);

/* Secret key coefficients (ternary, N values) to the host. */
copse_status copse_keys_export_secret(const copse_keys *keys, int64_t *s);

/* A switching key in coefficient form to the host, layout
 * [digit][2][n_primes + alpha][N] (words = digits * 2 * (L+alpha) * N).
 * galois = 0 selects the relinearisation key, else the key of that Galois
 * element (3^k mod 2N for a rotation by k).  ENOKEY if absent. */
copse_status copse_evk_export(const copse_evk *evk, uint64_t galois, uint64_t *out, size_t words);

/* ---------------------------------------------------------------- data */

/* Encrypt n_queries feature vectors for `model` (Section 3.3, Step 0):
 * each feature is replicated K times, laid out periodically in the query's
 * slot block, split into `precision` bit-planes (Section 4.1.2) and each plane
 * encrypted under the public key with randomness from `seed` (plane i uses
 * encryption index i).  feats[n_queries * n_features], values < 2^precision,
 * host memory if feats_on_device = 0, else device memory.  At most
 * N / block queries.  The new buffer holds `precision` ciphertexts.
 * Async on `stream` when feats_on_device = 1. */
copse_status copse_encrypt_features(copse_ctx *ctx, const copse_keys *keys, copse_model *model,
                                    const uint32_t *feats, size_t n_queries, int feats_on_device, uint64_t seed,
                                    copse_ctbuf **out, void *stream);

/* Secure inference, Algorithm 1 (Section 4.3): SecComp, reshuffle, level
 * products with masks, product across levels.  `feats` comes from
 * copse_encrypt_features for the same model.  Output: one ciphertext whose
 * slot block j holds query j's leaf bits.  Async on `stream`. */
copse_status copse_infer(copse_ctx *ctx, const copse_evk *evk, copse_model *model, const copse_ctbuf *feats,
                         copse_ctbuf **out, void *stream);

/* copse_infer with the per-step breakdown that Section 8.4 reports for the
 * Table 6 microbenchmarks: CUDA events recorded on `stream` at the step
 * boundaries give stage_ms[0] comparison (SecComp, Section 4.1.2),
 * stage_ms[1] reshuffling (R * Decisions), stage_ms[2] level processing
 * (Lvl_k * Branches XOR Mask_k), stage_ms[3] aggregation (product across
 * levels).  The result is the same ciphertext copse_infer returns.  Blocks
 * the calling thread until the stream reaches the end of the inference;
 * EINVAL while a graph is being recorded on the context, or on null
 * arguments; stage_ms is host memory owned by the caller. */
copse_status copse_infer_timed(copse_ctx *ctx, const copse_evk *evk, copse_model *model, const copse_ctbuf *feats,
                               copse_ctbuf **out, void *stream, float stage_ms[4]);

/* Decrypt an inference result into out_bits[n_queries * n_leaves]: 1 for the
 * leaf each tree selects, 0 elsewhere, 2 for a slot that is not a bit
 * (noise overflow).  out_bits is host memory if out_on_device = 0 (the call
 * then synchronises), else device memory (async). */
copse_status copse_decrypt_labels(copse_ctx *ctx, const copse_keys *keys, const copse_model *model,
                                  const copse_ctbuf *result, uint8_t *out_bits, size_t n_queries,
                                  int out_on_device, void *stream);

/* All N slot values (mod t, slot order: row 0 columns 0..N/2-1, then row 1)
 * of ciphertext `index`, to host memory out_slots[N].  Synchronous. */
copse_status copse_decrypt_slots(copse_ctx *ctx, const copse_keys *keys, const copse_ctbuf *buf, size_t index,
                                 uint64_t *out_slots);

/* ---------------------------------------------------------------- sessions
 * A session fixes the context, keys, model and number of queries and records
 * one whole secure inference -- feature encryption (Section 3.3, Step 0),
 * Algorithm 1 (Section 4.3) and decryption of the leaf bits -- as a CUDA
 * graph, replayed by every run.  The same per-model operation sequence is
 * reused for every batch of queries; results equal copse_encrypt_features +
 * copse_infer + copse_decrypt_labels with the same seed. */
typedef struct copse_session copse_session;

/* Record the graph (uploads the model's plaintexts first; synchronous).
 * n_queries <= N / block.  keys, evk and model must outlive the session. */
copse_status copse_session_create(copse_ctx *ctx, const copse_keys *keys, const copse_evk *evk,
                                  copse_model *model, size_t n_queries, copse_session **out);
/* A session over n_items work items (models[i], n_queries[i]): one graph
 * launch evaluates every item, each on its own lane of streams, so queries of
 * several forests of uneven size run in one launch.  Runs take the items'
 * features concatenated in item order and return their leaf bits
 * concatenated in item order; item i encrypts with seed + i.  A model may
 * appear in several items (each item holds up to N / block queries). */
copse_status copse_session_create_batch(copse_ctx *ctx, const copse_keys *keys, const copse_evk *evk,
                                        size_t n_items, copse_model *const *models, const size_t *n_queries,
                                        copse_session **out);
/* One step: feats[n_queries * n_features] (host if feats_on_device = 0, else
 * device), fresh encryption randomness from `seed`, leaf bits into
 * out_bits[n_queries * n_leaves] (host if out_on_device = 0: the call then
 * synchronises; else device: async).  Runs on `stream`; runs of one session
 * must not overlap (they share the session's buffers). */
copse_status copse_session_run(copse_session *session, const uint32_t *feats, int feats_on_device, uint64_t seed,
                               uint8_t *out_bits, int out_on_device, void *stream);
void copse_session_destroy(copse_session *session);

/* ---------------------------------------------------------------- serving
 * The evaluator of the paper's workflow (Section 3.2: the server accepts
 * inference queries against resident models) as a request loop.  Each request
 * is one query for one model.  A worker thread packs a model's pending
 * requests into the slot blocks of that model's next launch (continuous
 * batching: requests that arrive while a launch is on the GPU join the next
 * one) and keeps up to two launches per model in flight.  Keys, model
 * plaintexts and the launches' device memory stay resident.  Admission is by
 * device memory: creation measures each launch's reservation (the peak of
 * graph-allocated device memory while its graph is replayed once), gives a model
 * its second concurrent launch only while free memory holds another such
 * reservation plus the admission floor, and fails with COPSE_EADMIT when not
 * even one launch per model fits.  A request is then admitted only while free
 * device memory is at least the floor (default: the largest launch
 * reservation, room for one more launch's working set) and the pending queue
 * holds fewer than max_pending requests (0 = four times the slot capacity of
 * all launches).  The server is internally locked. */
typedef struct copse_server copse_server;

copse_status copse_server_create(copse_ctx *ctx, const copse_keys *keys, const copse_evk *evk,
                                 copse_model *const *models, size_t n_models, size_t max_pending,
                                 copse_server **out);
/* Queue one query (feats[n_features], host) for models[model_id].  Returns a
 * ticket, or COPSE_EADMIT when free device memory is below the admission floor
 * or the queue is full (nothing queued). */
copse_status copse_server_submit(copse_server *server, uint32_t model_id, const uint32_t *feats, uint64_t *ticket);
/* Wait up to timeout_ms for a ticket: its leaf bits into out_bits[n_leaves]
 * (host) and, if latency_ms is not NULL, the time from submit to completion.
 * COPSE_ETIMEOUT if not ready (the ticket stays valid); a ticket is released
 * by the successful poll, so another poll of it (also one that was waiting in
 * another thread) fails with COPSE_EINVAL. */
copse_status copse_server_poll(copse_server *server, uint64_t ticket, uint8_t *out_bits, int timeout_ms,
                               double *latency_ms);
/* Device memory of the server: bytes its launches reserved at creation, the
 * largest single launch's reservation, the current admission floor (free
 * device bytes a submit requires) and the number of concurrent launches all
 * models together were given.  Any pointer may be NULL. */
copse_status copse_server_memory(copse_server *server, size_t *reserved, size_t *launch_max, size_t *floor,
                                 uint32_t *launches);
/* Set the admission floor: submits fail with COPSE_EADMIT while free device
 * memory is below `floor` bytes (0 = admit regardless of memory). */
copse_status copse_server_set_memory_floor(copse_server *server, size_t floor);
/* Requests waiting for a launch, and requests in launches on the GPU. */
copse_status copse_server_pending(copse_server *server, size_t *queued, size_t *in_flight);
/* Stops the worker after the launches in flight and frees everything. */
void copse_server_destroy(copse_server *server);

/* ---------------------------------------------------------------- buffers */

size_t copse_ctbuf_count(const copse_ctbuf *buf);
/* Level (primes) and components of ciphertext `index`. */
copse_status copse_ctbuf_shape(const copse_ctbuf *buf, size_t index, uint32_t *level, uint32_t *ncomp);
/* Ciphertext `index` in coefficient form to the host, layout
 * [component][prime][N], residues in [0, q_i).  Synchronous. */
copse_status copse_ctbuf_export(copse_ctx *ctx, const copse_ctbuf *buf, size_t index, uint64_t *out, size_t words);
/* New buffer of n_ct two-component ciphertexts at `level` from coefficient
 * form host data, layout [ct][2][level][N].  Synchronous. */
copse_status copse_ctbuf_import(copse_ctx *ctx, const uint64_t *in, size_t n_ct, uint32_t level,
                                copse_ctbuf **out);
void copse_ctbuf_destroy(copse_ctbuf *buf);

/* ---------------------------------------------------------------- ring ops
 * Single BGV operations on buffer entries, for per-operation checks.  All
 * create a new one-ciphertext buffer and are async on `stream`. */

/* a * b, relinearised, then one prime dropped (the multiply of Section 6). */
copse_status copse_ct_mul(copse_ctx *ctx, const copse_evk *evk, const copse_ctbuf *a, size_t ia,
                          const copse_ctbuf *b, size_t ib, copse_ctbuf **out, void *stream);
/* Rotation of every slot row left by k (Section 4.1.2, Matrix Multiplication). */
copse_status copse_ct_rotate(copse_ctx *ctx, const copse_evk *evk, const copse_ctbuf *a, size_t ia, uint32_t k,
                             copse_ctbuf **out, void *stream);
/* Drop the last prime. */
copse_status copse_ct_modswitch(copse_ctx *ctx, const copse_ctbuf *a, size_t ia, copse_ctbuf **out, void *stream);
/* a * plaintext + plaintext: slot vectors mul_slots[N], add_slots[N] (host,
 * values mod t; add_slots may be NULL). */
copse_status copse_ct_mul_plain(copse_ctx *ctx, const copse_ctbuf *a, size_t ia, const uint64_t *mul_slots,
                                const uint64_t *add_slots, copse_ctbuf **out, void *stream);

/* Forward (inverse = 0) or inverse negacyclic NTT, in place, of n_polys
 * polynomials laid out [n_polys][n_res][N] in device memory, residue r taken
 * modulo ciphertext prime r (n_res <= n_primes).  Coefficient order in,
 * bit-reversed evaluation order out (and back).  Async. */
copse_status copse_ntt(copse_ctx *ctx, uint64_t *data, size_t n_polys, uint32_t n_res, int inverse, void *stream);

/* Negacyclic product c = a * b in Z_q[X]/(X^N + 1), coefficient form in and
 * out, n_res residues per operand laid out [n_res][N] in device memory,
 * residue r modulo ciphertext prime r.  Uses temporary device memory from
 * the context's pool.  Async. */
copse_status copse_poly_mul(copse_ctx *ctx, const uint64_t *a, const uint64_t *b, uint64_t *c, uint32_t n_res,
                            void *stream);

/* The same product as copse_poly_mul, computed without allocating anything.
 * The paper has no counterpart: this exists for callers that cannot allocate
 * device memory when they need the product -- serving loops that forbid
 * allocation after start-up to keep latency flat and memory use fixed, or
 * programs whose device memory is already reserved by another allocator.
 * It calls no cudaMalloc, cudaFree or allocating library routine.
 * The caller still provides a, b and c (device memory, as for
 * copse_poly_mul).  The two transform buffers are a fixed device array of
 * 2 x 2^18 words (4 MiB) that every GPU loading this library holds until the
 * process exits; n_res * N above 2^18 words fails with COPSE_EINVAL.  The
 * context's device must be current on every call (COPSE_EINVAL otherwise).
 * The first call on a device looks up the array's device address; make that
 * first call before any stream capture.
 * All calls on a device share the array: calls that overlap on the GPU race,
 * so order them on one stream.  Async. */
copse_status copse_poly_mul_noalloc(copse_ctx *ctx, const uint64_t *a, const uint64_t *b, uint64_t *c,
                                    uint32_t n_res, void *stream);

/* ---------------------------------------------------------------- autotuning
 * The paper fixes its HElib parameters by hand (Section 8.1); these calls pick
 * schedule choices by running every candidate on the device and timing it
 * with CUDA events (median of `reps` timed runs after one warm-up).  None
 * changes a result: any choice gives a correct inference, the ciphertexts
 * differ only in rounding.  All block the calling thread. */

/* NTT kernel family by batch size: one thread-block-cluster launch per
 * transform against two tiled launches, forward + inverse of sizes[i]
 * residue polynomials each (ms_cluster[i], ms_tiled[i]).  The context then
 * takes the cluster form for batches up to *max_cluster residue polynomials
 * (the largest timed size at which it is not slower; 0 = never, 2^30 =
 * always, when that is the largest size timed) and the tiled form above. */
copse_status copse_tune_ntt(copse_ctx *ctx, const uint32_t *sizes, size_t n, int reps, float *ms_cluster,
                            float *ms_tiled, uint32_t *max_cluster);
/* Set the crossover copse_tune_ntt would choose (to replay a tuned schedule). */
copse_status copse_ctx_set_ntt_cluster_max(copse_ctx *ctx, uint32_t max_cluster);

/* The crossover of the forward / inverse transforms fused with the base
 * conversions around them (modulus switch, ModUp, ModDown): a fused launch
 * replaces a conversion kernel, a transform and a finishing kernel, so its
 * best crossover differs from the plain one.  Each cands[i] (residue
 * polynomials per launch; >= 2^30 = always) is set in turn and one whole
 * inference of the model's current plan timed (ms[i], median of reps); the
 * fastest stays set and is returned in *best.  Keys are made internally.
 * Fused transforms exist for 2^12 <= N <= 2^14; at other degrees nothing is
 * timed (ms[i] = -1) and *best is the current setting. */
copse_status copse_tune_fused(copse_ctx *ctx, copse_model *model, const uint32_t *cands, size_t n,
                              size_t n_queries, int reps, float *ms, uint32_t *best);
/* Set the fused crossover copse_tune_fused would choose (default: always fused). */
copse_status copse_ctx_set_ntt_fused_max(copse_ctx *ctx, uint32_t max_fused);

/* Baby-step sizes (copse_model_set_bsgs): the reshuffle candidates g_r[] are
 * timed by the reshuffle stage with the level plan held, then the level
 * candidates g_l[] by the level stage with the chosen reshuffle plan, each
 * with fresh keys for its plan and n_queries random queries.  ms_r[i], ms_l[i]:
 * stage medians, -1 for a candidate the query block cannot hold.  Leaves the
 * best plan set on the model; keys must then be made for it. */
copse_status copse_tune_bsgs(copse_ctx *ctx, copse_model *model, const uint32_t *g_r, size_t n_r,
                             const uint32_t *g_l, size_t n_l, size_t n_queries, int reps, float *ms_r,
                             float *ms_l);

/* Key-switching digit count: one context per candidate dnums[i] (base's other
 * parameters), one whole inference timed on each; ms[i] its median (-1 for a
 * parameter set out of range), *best the fastest dnum. */
copse_status copse_tune_dnum(const copse_params *base, int device, copse_model *model, const uint32_t *dnums,
                             size_t n, size_t n_queries, int reps, float *ms, uint32_t *best);

/* ---------------------------------------------------------------- kernel timing
 * Instrumentation, off by default.  When on, the library brackets every
 * kernel launch with two CUDA events on the launch stream and tags it with
 * its family (transforms: "ntt_fwd", "ntt_inv", "ntt_inv_copy" and the fused
 * forms "ntt_fwd_ms", "ntt_fwd_md", "ntt_fwd_mu", "ntt_fwd_mdd"; key switching
 * and products: "modup", "ks_inner", "mm_fused", "mm_finish", "rotsum",
 * "sum_parts", "enc_mac", "moddown_conv", "ks_finish", "ms_conv", "ms_finish";
 * elementwise: "tensor", "affine", "add") and its algorithmic bytes (each
 * operand read once, each result written once).  The paper's own measurement is per-stage wall time
 * (Section 8.4); this gives the per-kernel view. */
copse_status copse_stats_enable(int on);
/* Wait for the device and clear every total. */
copse_status copse_stats_reset(void);
/* Wait for the device; totals of family `name` (NULL or "" = all families):
 * launches, summed event time in milliseconds, algorithmic bytes. */
copse_status copse_stats_get(const char *name, uint64_t *launches, double *ms, double *bytes);
/* Wait for the device; algorithmic modular products of family `name` (NULL or
 * "" = all families): the 64-bit residue products the launches' method needs
 * (a ciphertext tensor counts 4 per element), the unit of the integer roof. */
copse_status copse_stats_get_ops(const char *name, double *ops);
/* Newline-separated family names seen so far into buf[cap]. */
copse_status copse_stats_names(char *buf, size_t cap);

/* ---------------------------------------------------------------- work lists
 * Many independent or chained elementwise ciphertext operations in one
 * persistent launch: as many CTAs as the device holds at once take the items'
 * tiles in list order; an item waits for the items it depends on, each wait
 * bounded by timeout_ms of the GPU's global timer.  (The encrypted-threshold
 * comparison leaves of Section 4.1.2 run through the same kernel.)  Item i's
 * operands a, b index `in` (r < count(in)) or the outputs of earlier items
 * (r = count(in) + j, j < i), all two-component ciphertexts at one level; its
 * result is ciphertext i of the new buffer *out:
 *   COPSE_WL_ADD a + b, COPSE_WL_SUB a - b, COPSE_WL_TENSOR the 3-component
 *   product (a0 b0, a0 b1 + a1 b0, a1 b1) before relinearisation.
 * An item waits for every earlier output it reads and, when dep >= 0, also for
 * item dep.  A list that waits for an item that cannot finish (dep naming the
 * item itself, or a later one that no running CTA reaches) runs into the limit:
 * the launch stops and the call returns COPSE_ETIMEOUT (no buffer made; the
 * context stays usable).  At most 256 items; timeout_ms >= 1.  Synchronous. */
#define COPSE_WL_ADD 0
#define COPSE_WL_SUB 1
#define COPSE_WL_TENSOR 3
typedef struct copse_wl_item {
    uint32_t kind;
    uint32_t a, b;  /* operands: index into `in`, or count(in) + an earlier item */
    int32_t dep;    /* an item to wait for besides the outputs read, -1 none  */
} copse_wl_item;
copse_status copse_worklist_run(copse_ctx *ctx, const copse_ctbuf *in, const copse_wl_item *items, size_t n,
                                int timeout_ms, copse_ctbuf **out, void *stream);

/* ---------------------------------------------------------------- integer peaks
 * The roofline of integer kernels needs a measured rate of the modular
 * arithmetic they are made of, not a spec-sheet figure.  Register-only
 * microbenchmarks on the context's device, CUDA-event timed, best of `reps`
 * runs after one warm-up run:
 *   kind 0: exact products x*y of residues below 2^55 added to a lazily reduced
 *           sum (split 28-bit multiply-adds), the unit of the dot-product kernels;
 *   kind 1: lazy forward NTT butterflies with a constant twiddle (Shoup/Harvey);
 *   kind 2: Barrett products of two residues, fully reduced.
 * *ops_per_s: products (kind 0, 2) or butterflies (kind 1) per second over the
 * whole device; *best_ms (may be NULL) the best run.  Allocates a small sink
 * buffer; synchronous.  EINVAL on a bad kind or reps < 1. */
copse_status copse_measure_int_peak(copse_ctx *ctx, int kind, int reps, double *ops_per_s, float *best_ms);

#ifdef __cplusplus
}
#endif

#endif /* COPSE_H */
