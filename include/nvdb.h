/*
 * nvdb.h -- C ABI of libnvdb.so, a B300 (sm_103a) implementation of the
 * NeuralVDB hot path (Kim, Lee & Museth, "NeuralVDB: High-resolution Sparse
 * Volume Representation using Hierarchical Neural Networks").
 *
 * NeuralVDB keeps the root and level-2 nodes of a VDB [Hash,5,4,3] tree
 * explicit and replaces the two lower levels by coordinate networks
 * (Section 3.3.1): a level-1 mask classifier, a level-0 (voxel) mask
 * classifier and a voxel value regressor, each a Fourier-feature encoding
 * (Section 3.2.2, Eq. 2) followed by a ReLU MLP.  Misclassified candidates are
 * stored as patches (Section 3.3.2), so decoding restores the topology
 * exactly; values are lossy.
 *
 * Conventions for every call:
 *  - Pointers named d_* are DEVICE pointers (CUDA global memory of the current
 *    device); every other pointer is a HOST pointer.  The caller owns all
 *    buffers it passes; the library owns the nvdb_grid / nvdb_model handles
 *    (free them with nvdb_grid_free / nvdb_model_free) and the device memory
 *    inside them.
 *  - Work is enqueued on the given stream and ordered with it.  Calls that
 *    return counts or device-detected errors synchronise that stream before
 *    returning; the others (noted per call) return without synchronising.
 *  - No C++ exception crosses this boundary.  A call returns NVDB_OK or an
 *    error status; nvdb_last_error() gives a message for the calling thread.
 *  - Voxel coordinates are int32 triples (i, j, k) in [0, 2^21).
 *  - Mask bits: bit b of a node mask is bit (b & 63) of 64-bit word (b >> 6).
 *    Slot / offset numbering follows the dense VDB node layout (Section 3.1):
 *    level-2 slot = ((i>>7)&31)<<10 | ((j>>7)&31)<<5 | ((k>>7)&31),
 *    leaf slot    = ((i>>3)&15)<<8  | ((j>>3)&15)<<4 | ((k>>3)&15),
 *    voxel offset = (i&7)<<6 | (j&7)<<3 | (k&7).
 *    Canonical voxel order is lexicographic on (level-2 origin, level-1 slot,
 *    leaf slot, voxel offset).
 */
#ifndef NVDB_H
#define NVDB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* nvdb_stream;   /* a cudaStream_t; NULL = legacy default stream */

typedef enum {
  NVDB_OK = 0,
  NVDB_ERR_INVALID_ARG = 1,     /* NULL pointer, bad size, coordinate out of range, unknown option */
  NVDB_ERR_DUPLICATE_VOXEL = 2, /* nvdb_build: the same (i,j,k) appears twice */
  NVDB_ERR_OUT_OF_MEMORY = 3,   /* a device or host allocation failed */
  NVDB_ERR_CAPACITY = 4,        /* caller's output buffer too small; counts hold the need */
  NVDB_ERR_CUDA = 5,            /* a CUDA runtime call failed (message names it) */
  NVDB_ERR_TIMEOUT = 6,         /* a device-side wait gave up (bounded spin) */
  NVDB_ERR_UNSUPPORTED = 7,     /* valid but not implemented (width, precision, ...) */
  NVDB_ERR_CORRUPT = 8          /* blob or decoded counts inconsistent with the model header */
} nvdb_status;

/* Arithmetic of the hidden layers when evaluating networks. */
typedef enum {
  NVDB_FP32 = 0,      /* plain FP32 on CUDA cores (FFMA), FP32 encoding */
  NVDB_BF16 = 1,      /* tcgen05 tensor cores, BF16 operands (one MMA term), FP32 accumulate in TMEM */
  NVDB_FP8_E4M3 = 2,  /* tcgen05: first layer FP16 on the encoding, hidden layers E4M3 activations
                         and weights (kind::f8f6f4) with one scale per layer, FP32 accumulate */
  NVDB_FP16 = 3,      /* tcgen05 tensor cores, FP16 operands (one MMA term), FP32 accumulate in TMEM */
  NVDB_BF16X3 = 4     /* tcgen05 tensor cores, activations and weights as hi + lo BF16 pairs
                         (three MMA terms; two when the weights are BF16 values), FP32 accumulate */
} nvdb_precision;

/* Network indices (Section 3.3.1).  A model of a grid with active tiles (nvdb_build_opts
 * prune_tiles) has a fourth network, the tile value regressor, and its level-1 classifier is
 * ternary: three logits per slot for the classes child leaf (0), active tile (1) and
 * inactive (2), the class the first maximum. */
enum { NVDB_NET_L1_CLASSIFIER = 0, NVDB_NET_L0_CLASSIFIER = 1, NVDB_NET_REGRESSOR = 2, NVDB_NET_TILE_REGRESSOR = 3 };
/* Hidden activations (the activation appendix and the hyper-parameter table). */
enum { NVDB_ACT_RELU = 0, NVDB_ACT_SIN = 1 /* sin(omega a) */ };
/* Losses (Eq. 1 is MSE; BCE is used for the classifiers, Section 3.3.1). */
enum { NVDB_LOSS_MSE = 0, NVDB_LOSS_L1 = 1, NVDB_LOSS_BCE = 2,
       NVDB_LOSS_LINEAR = 3 /* nvdb_mlp_grad only: d_target holds dL/dy per sample; the gradient is
                               sum_s target_s dy_s/dtheta (a vector-Jacobian product) */,
       NVDB_LOSS_CE = 4     /* softmax cross-entropy of the ternary classifier's three logits
                               (Section 3.3.1); the target is the class 0, 1 or 2 as a float */ };

typedef struct nvdb_grid nvdb_grid;    /* explicit [Hash,5,4,3] tree, device resident */
typedef struct nvdb_model nvdb_model;  /* [Hash,5,NN(4),NN(3)]: upper tree + 3 networks + patches */

typedef struct {
  int32_t grid_class;   /* 0 = narrow-band level set (SDF), 1 = fog (density) */
  float half_width;     /* level sets: band half-width w in voxels (values lie in (-w, w)); fog: ignored */
  int32_t prune_tiles;  /* 1: tile pruning (Section 3.1) -- a leaf whose 512 voxels are all active and
                           whose values span at most tile_tolerance (FP32 max - min) becomes an active
                           tile of its level-1 node with the FP32 midpoint (min + max) / 2 as value;
                           the grid keeps it expanded as its leaf, every voxel carrying the tile value.
                           0: every voxel stays explicit */
  float tile_tolerance; /* >= 0 */
} nvdb_build_opts;

typedef struct {
  uint64_t seed;        /* seeds the initial weights, the Fourier matrix and the sample stream */
  int32_t width[3];     /* hidden width per network (supported: 32, 64) */
  int32_t layers[3];    /* hidden layers per network (1..8) */
  int32_t ffm_size[2];  /* encoding size n of level 1 and level 0 (supported: 32, 64); 0 = max width */
  float ffm_sigma;      /* std of the Fourier matrix B, in cycles over the domain extent E */
  int32_t steps;        /* Adam steps per network */
  int32_t batch;        /* samples per step (uniform with replacement, Section 3.2.1) */
  float lr;             /* learning rate */
  float lr_decay;       /* gamma: lr_t = lr * gamma^floor((t-1)/lr_interval) */
  int32_t lr_interval;  /* 0 = constant learning rate */
  int32_t loss;         /* regressor loss: NVDB_LOSS_MSE or NVDB_LOSS_L1 */
  int32_t train_prec;   /* arithmetic of training: NVDB_FP32 or NVDB_BF16 (tensor cores) */
  uint32_t patch_precs; /* bit p set = store patches for decoding at precision p (default: all five) */
  int32_t stop_window;  /* early stop (warm-started frames, Section 3.6): every stop_window steps ... */
  float stop_loss[3];   /* ... network k stops once the mean of its last stop_window losses < stop_loss[k];
                           0 = train all `steps` */
  int32_t resume;       /* with a warm model: continue its training (checkpoint / resume) -- its FP32
                           master weights, Adam moments and step count, so that `steps` more steps
                           equal the same steps of an uninterrupted run bit for bit (same options;
                           the warm model must have been trained in this process, since exported
                           blobs carry no Adam state); 0 = warm start (weights only, Section 3.6) */
  int32_t subdomain;    /* sparse domain decomposition (Section 3.4): subdomain size S in voxels, a
                           multiple of 512; 0 = none (one network per level over the whole domain).
                           Subdomains of a regular grid from the domain origin that hold voxels keep
                           an expert each (the three networks, normalised over the subdomain); a
                           point's output is the gate-weighted average of the experts whose clamped
                           tent gate (subdomain plus halo) is non-zero there (Eq. 3).  A warm start
                           takes the warm model's decomposition. */
  int32_t halo;         /* halo width in voxels, a power of two in [8, S/4]; 0 = 8 */
  int32_t resample;     /* subset resampling (Appendix E): every `resample` steps draw a subset of
                           resample x batch candidates, and each step's batch from that subset;
                           0 = a fresh batch every step (resample x batch < 2^32) */
  int32_t sampling;     /* regressor samples (Appendix C ablation): 0 = active voxels (the method),
                           1 = every voxel of the leaves (blocked), 2 = every voxel of the domain's
                           bounding box (dense; log2 extent <= 10, no decomposition); inactive
                           voxels take the background as target */
  int32_t activation;   /* hidden activation of every network: NVDB_ACT_RELU, or NVDB_ACT_SIN (sin(omega a):
                           FP32 training; evaluation at FP32, FP16, BF16, BF16X3 but not FP8, so
                           patch_precs must leave out FP8; with a decomposition FP32 only) */
  float omega;          /* sin frequency (the paper's 1.5 .. 3.0) */
  int32_t tile_width;   /* grids with active tiles: tile value regressor width (0 = width[0]) ... */
  int32_t tile_layers;  /* ... and hidden layers (0 = layers[0]); it and the ternary level-1
                           classifier train at train_prec like the other networks (the classifier
                           evaluates at every precision) */
} nvdb_train_opts;

typedef struct {
  int32_t grid_class;
  float background, half_width;
  int32_t origin[3];     /* encoding domain origin (multiple of 128) */
  int32_t log2_extent;   /* encoding domain extent E = 2^log2_extent voxels */
  int64_t n_active, n_leaf, n_l1, n_l2;
  int32_t n_experts;     /* models: experts of the domain decomposition (1 without one); grids: 0 */
  int32_t subdomain;     /* models: subdomain size S (0 = no decomposition) */
  int64_t n_tiles;       /* active tiles of level 1 (grids built with prune_tiles, and their models) */
} nvdb_info;

/* ------------------------------------------------------------------------ */

/* Build the explicit VDB [Hash,5,4,3] tree (Section 3.1, Fig. 1) from n sparse
 * voxels: d_ijk int32 [n][3], d_val float [n], any order.  The grid copies the
 * voxels in canonical order plus leaf/level-1/level-2 origins and masks.
 * Errors: INVALID_ARG (n < 0, NULL, coordinate outside [0,2^21)),
 * DUPLICATE_VOXEL.  Synchronises the stream (node counts size the tree). */
nvdb_status nvdb_build(const int32_t* d_ijk, const float* d_val, int64_t n,
                       const nvdb_build_opts* opts, nvdb_stream stream, nvdb_grid** out);

nvdb_status nvdb_grid_info(const nvdb_grid* grid, nvdb_info* out);

/* Copy the grid's canonical arrays to HOST buffers (any pointer may be NULL):
 * ijk [n][3], val [n], leaf_origin [n_leaf][3], leaf_mask [n_leaf][8],
 * l1_origin [n_l1][3], l1_mask [n_l1][64].  Synchronises the stream. */
nvdb_status nvdb_grid_read(const nvdb_grid* grid, int32_t* ijk, float* val, int32_t* leaf_origin,
                           uint64_t* leaf_mask, int32_t* l1_origin, uint64_t* l1_mask,
                           nvdb_stream stream);

/* The grid's active tiles to HOST buffers (either may be NULL): leaf_tile [n_leaf] (1 = the
 * leaf is an active tile), l1_tile_mask [n_l1][64] (the level-1 active masks a_1).  Zero for a
 * grid built without tile pruning.  Synchronises the stream. */
nvdb_status nvdb_grid_tiles(const nvdb_grid* grid, uint8_t* leaf_tile, uint64_t* l1_tile_mask, nvdb_stream stream);

nvdb_status nvdb_grid_free(nvdb_grid* grid);

/* Point samples of the explicit grid (the comparison samplers of Section 4.4): order 0 the
 * value of the voxel nearest p (floor(p + 1/2)), 1 trilinear over the cell's 8 corners
 * (corner c = 4a + 2b + d, weight (wx wy) wz), 3 Catmull-Rom tricubic over the 4^3 voxels
 * around the cell; inactive voxels take the background (+half_width for level sets, 0 for
 * fog).  d_xyz float [n][3] (index space), d_out float [n].  The first call builds the
 * grid's random-access structures (keys, per-word popcount prefixes, child bases) and
 * synchronises; later calls do not. */
nvdb_status nvdb_grid_sample(const nvdb_grid* grid, const float* d_xyz, int64_t n, int order, float* d_out,
                             nvdb_stream stream);

/* Zero crossings of a level-set grid along the +x, +y, +z edges of its active voxels whose
 * neighbour is active with the other sign (the isosurface points of Eq. 4's mCD): v + t e_a,
 * t = val(v) / (val(v) - val(v + e_a)), in canonical voxel order then axis order.  With
 * d_pts NULL only *count is set; else d_pts float [capacity][3] (CAPACITY if too small).
 * Synchronises the stream. */
nvdb_status nvdb_grid_isosurface(const nvdb_grid* grid, float* d_pts, int64_t capacity, int64_t* count,
                                 nvdb_stream stream);

/* Modified Chamfer distance (Eq. 4) between a reference and a reconstructed level set:
 * mCD = 1/(2 N1) sum_i |SDF_rec(v1_i)| + 1/(2 N2) sum_i |SDF_ref(v2_i)|, v1 / v2 the
 * isosurface points of the reference / reconstruction (nvdb_grid_isosurface), each SDF
 * sampled trilinearly from the other grid (nvdb_grid_sample, order 1).  *mcd (HOST) in
 * voxels.  Synchronises the stream. */
nvdb_status nvdb_mcd(const nvdb_grid* reference, const nvdb_grid* reconstruction, double* mcd, nvdb_stream stream);

/* Fill opts with the defaults: widths 32, 3 layers, ffm_size 0, sigma 1.25,
 * 200 steps, batch 4096, lr 1e-3, decay 0.975 every 100 steps, MSE, FP32
 * training, patches for FP32, BF16 and FP16, seed 1, no early stop (window 50). */
void nvdb_train_opts_default(nvdb_train_opts* opts);

/* Encode a grid (Sections 3.2-3.3): initialise the three networks (Xavier
 * weights and the Fourier matrix B ~ N(0, sigma^2), drawn from SplitMix64
 * streams of opts->seed) or copy them from `warm` (temporally coherent warm
 * start, Section 3.6; warm may be NULL), train each for opts->steps Adam steps
 * on uniformly sampled candidates (Philox4x32-10 sample stream; regressor on
 * active voxels only, Section 3.2.1), then classify every candidate at each
 * precision of opts->patch_precs and store the mismatches as patches
 * (Section 3.3.2).  Synchronises the stream. */
nvdb_status nvdb_compress(const nvdb_grid* grid, const nvdb_train_opts* opts, const nvdb_model* warm,
                          nvdb_stream stream, nvdb_model** out);

/* Animated volumes (Section 3.6, temporally coherent warm start): encode frames 0..n-1 of a
 * sequence into out[0..n-1].  Frame 0 is trained cold with `opts`, then refined from those
 * weights for refine_steps steps at lr x refine_lr_scale (fresh Adam state; 0 steps = no
 * refinement); frame 0's final loss per network is the mean of its last opts->stop_window
 * losses.  Every later frame starts from the previous frame's networks and Fourier matrices
 * and trains at lr x refine_lr_scale for at most warm_steps steps, each network stopping at
 * the first multiple of stop_window steps whose last stop_window losses average below frame
 * 0's final loss.  Models are owned by the caller (nvdb_model_free); on an error none is
 * returned.  Synchronises the stream. */
nvdb_status nvdb_compress_sequence(const nvdb_grid* const* grids, int n_frames, const nvdb_train_opts* opts,
                                   float refine_lr_scale, int32_t refine_steps, int32_t warm_steps,
                                   nvdb_stream stream, nvdb_model** out);

/* Per-step mean training loss of network `net` of the last compress
 * (HOST buffer of cap floats); *count receives the number of steps run
 * (fewer than opts->steps when the early stop triggered). */
nvdb_status nvdb_model_losses(const nvdb_model* model, int net, float* losses, int64_t cap,
                              int64_t* count);

/* Decode models back to voxels (Section 3.5, offline sequential access; Fig. 5):
 * level-1 node origins from the level-2 child masks, level-1 classification +
 * patches -> child leaves, level-0 classification + patches -> active voxels,
 * regression of the active voxels -> values (x half_width for level sets).
 * Outputs are concatenated per model in canonical order: d_ijk int32 [cap][3],
 * d_val float [cap]; counts (HOST, n_models entries) receives each model's
 * active count.  If d_ijk is NULL only counts are filled (from the headers).
 * Errors: CAPACITY (sum of counts > capacity; nothing written), UNSUPPORTED
 * (no patch set for prec), CORRUPT (decoded counts differ from the header).
 * Synchronises the stream. */
nvdb_status nvdb_decompress(const nvdb_model* const* models, int n_models, nvdb_precision prec,
                            int32_t* d_ijk, float* d_val, int64_t capacity, int64_t* counts,
                            nvdb_stream stream);

/* nvdb_decompress with the result delivered to HOST memory as well: the
 * voxels are decoded into d_ijk / d_val as above and copied to h_ijk int32
 * [cap][3] / h_val float [cap] (caller-owned; page-locked memory lets the
 * copies run asynchronously).  The voxel copy starts as soon as the voxels
 * are emitted, on a stream of the library's own, and overlaps the
 * regression; the value copy follows it.  Returns when both copies have
 * landed.  h_ijk and h_val may be NULL only when d_ijk is (counts only).
 * Errors as nvdb_decompress. */
nvdb_status nvdb_decompress_host(const nvdb_model* const* models, int n_models, nvdb_precision prec,
                                 int32_t* d_ijk, float* d_val, int32_t* h_ijk, float* h_val,
                                 int64_t capacity, int64_t* counts, nvdb_stream stream);

/* Decode plan: the whole nvdb_decompress of `models` into the given output
 * buffers, recorded once into a CUDA graph (the benchmark spec: batched, graph-captured
 * decode).  Models with the same network shapes are decoded together, up to 48
 * per launch of each stage (levels, chunks and frames of several models share
 * one launch).  Building the plan runs the decode several times to pick the
 * number of tensor-core CTAs per SM (the autotuner; 0 = the kernel's own
 * limit), then captures it on `stream`.  The outputs are overwritten by every
 * launch.  Synchronises the stream. */
typedef struct nvdb_plan nvdb_plan;
nvdb_status nvdb_decompress_plan(const nvdb_model* const* models, int n_models, nvdb_precision prec,
                                 int32_t* d_ijk, float* d_val, int64_t capacity, nvdb_stream stream,
                                 nvdb_plan** out);
/* Replay the plan on `stream` (does not synchronise). */
nvdb_status nvdb_plan_launch(nvdb_plan* plan, nvdb_stream stream);
/* Synchronise `stream` and report device-detected errors of the last launch. */
nvdb_status nvdb_plan_check(nvdb_plan* plan, nvdb_stream stream);
/* Tuning result (HOST outputs, any may be NULL): tensor-core CTAs per SM chosen (0 = the
 * kernel's limit), the kernel variant chosen (0: 128 threads per tile; 1: 256 threads per
 * tile, each half of the accumulator columns in its own warps, node / leaf origins staged
 * by bulk copies; 2: 128 threads per tile with the origins staged by bulk copies two tiles
 * ahead), and the tuned decode time in ms. */
nvdb_status nvdb_plan_info(const nvdb_plan* plan, int* tc_ctas_per_sm, int* tc_variant, float* tuned_ms);
nvdb_status nvdb_plan_free(nvdb_plan* plan);

/* Random access on [Hash,5,4,NN(3)] (Section 3.5, online random access): for
 * each point p (float32 [n][3], index space) the 8 corners of the cell
 * floor(p) are looked up in the explicit topology (decoded once and cached in
 * the model); active corners are regressed, inactive corners take the
 * background (+half_width for level sets, 0 for fog); the result is the
 * trilinear blend with weights (w_x w_y) w_z, corners summed in the order
 * c = 4a + 2b + d for offset (a, b, d).  d_out float [n]; d_active (may be
 * NULL) uint8 [n] receives the active-corner bitmask (bit c).
 * FP32 does not synchronise unless the topology cache is built by this call;
 * the tensor-core precisions end with one stream synchronisation that reads
 * the model's device status word (NVDB_ERR_TIMEOUT if a bounded wait ran out).
 * Calls on one model that overlap on the GPU share that word. */
nvdb_status nvdb_query(const nvdb_model* model, const float* d_xyz, int64_t n, nvdb_precision prec,
                       float* d_out, uint8_t* d_active, nvdb_stream stream);

/* Pinhole camera of nvdb_render (index space). */
typedef struct {
  float eye[3];        /* camera position */
  float target[3];     /* point on the view axis */
  float up[3];         /* approximate up direction (not parallel to the view axis) */
  float fov_deg;       /* vertical field of view, (0, 180) */
  int32_t width, height;
  float step;          /* march step in voxels (> 0) */
  int32_t max_steps;   /* samples per ray, from the ray's entry into the domain box */
  float sigma;         /* extinction per unit density and voxel */
} nvdb_camera;

/* Ray-march a density model on [Hash,5,4,NN(3)] (Section 4, the ray-marched Bunny Cloud):
 * rays of a pinhole camera through pixel centres, clipped to the model's domain box; samples
 * at t_in + (k + 1/2) step, k < max_steps, while inside the box; the density at each sample
 * is nvdb_query's (trilinear over the regressed active corners, background elsewhere,
 * clamped at 0); emission-absorption composited front to back, alpha = 1 - exp(-sigma rho
 * step), L += T alpha rho, T *= 1 - alpha.  d_image float [height][width][2] = (L, T), a
 * headless device buffer.  Synchronises the stream. */
nvdb_status nvdb_render(const nvdb_model* model, const nvdb_camera* cam, nvdb_precision prec, float* d_image,
                        nvdb_stream stream);

/* Raw output (logit or unscaled value) of network `net` (0, 1, 2; 3 the tile value
 * regressor of a model with tiles) at n voxel coordinates d_ijk int32 [n][3]; the
 * level-1 networks take leaf origins (their input is ijk >> 3).  For a decomposed
 * model (Section 3.4) this is the gate-weighted average of its experts (Eq. 3), as
 * decoding uses it.  d_out float [n], or [n][3] (the three class logits) for the
 * ternary level-1 classifier.  Sin networks: no FP8.  FP32 does not synchronise; the
 * tensor-core precisions synchronise once to read the status word, as nvdb_query. */
nvdb_status nvdb_mlp_eval(const nvdb_model* model, int net, nvdb_precision prec, const int32_t* d_ijk,
                          int64_t n, float* d_out, nvdb_stream stream);

/* Gradient of the mean loss over n samples (d_ijk int32 [n][3], d_target
 * float [n]) w.r.t. the parameters of network `net` (Section 3.2), in the
 * arithmetic of one training step of precision `prec`: NVDB_FP32 (CUDA cores)
 * or NVDB_BF16 (tensor cores: BF16 operands, FP32 accumulation, FP32 head and
 * loss; at most 4 hidden layers; ReLU networks); other precisions return
 * NVDB_ERR_UNSUPPORTED.  The ternary classifier (three outputs) takes loss_kind
 * NVDB_LOSS_CE and class targets (0, 1, 2); another target value fails the call with
 * NVDB_ERR_INVALID_ARG (its rows are left out of the gradient); the other networks
 * take any other loss.
 * d_grad float [nvdb_net_param_count] in storage order (W_0, b_0, ...,
 * W_{L-1}, b_{L-1}, w_h, b_h; W row-major [out][in]); *loss (HOST) the mean
 * loss.  loss_kind: NVDB_LOSS_*.  Synchronises the stream. */
nvdb_status nvdb_mlp_grad(const nvdb_model* model, int net, nvdb_precision prec, const int32_t* d_ijk,
                          const float* d_target, int64_t n, int loss_kind, float* d_grad, float* loss,
                          nvdb_stream stream);

/* Same result as nvdb_mlp_grad, but allocates no device memory.  (The paper
 * has no counterpart; this exists for callers, not for the method.)  It is for
 * code that may not call cudaMalloc/cudaFree: applications whose device memory
 * is owned by their own pool or arena, and latency-critical loops where an
 * allocation, or the device-wide synchronisation a free can cause, is not
 * acceptable.  nvdb_mlp_grad keeps its gradient partials in memory the model
 * allocates on first use; this call keeps them, and the loss, in one static
 * device array of 2^20 floats (4 MiB) that every GPU loading the library holds
 * until the library is unloaded.
 *  - Every call looks the array's device address up with cudaGetSymbolAddress
 *    (which allocates nothing) on the current device; the first call on a device
 *    loads the library's device code there, so make it before any stream capture
 *    begins.  The library must not be used across a device reset of a live
 *    context it has worked in.
 *  - d_grad must hold nvdb_net_param_count(model, net) floats; the Python binding
 *    checks this, and the shapes of d_ijk and d_target, before any launch.
 *  - All calls share the array, and each call overwrites it (every block clears
 *    its own part before use).  Calls that can overlap on the GPU -- on
 *    different streams, or from different threads -- race on it; serialise them.
 *  - Limit: a network of more than 2^20 - 2 parameters is rejected with
 *    NVDB_ERR_CAPACITY.  Fewer thread blocks run than in nvdb_mlp_grad when the
 *    array cannot hold one partial per SM, so the summation order (and the
 *    last bits of the result) may differ.
 * Arguments, outputs and synchronisation as for nvdb_mlp_grad with NVDB_FP32. */
nvdb_status nvdb_mlp_grad_static(const nvdb_model* model, int net, const int32_t* d_ijk, const float* d_target,
                                 int64_t n, int loss_kind, float* d_grad, float* loss, nvdb_stream stream);

/* Network indices of the calls below (gradient, parameters, losses): network j of expert
 * e is 3e + j, so 0, 1, 2 without a domain decomposition; 0 <= net < 3 n_experts; a model
 * with tiles has net 3, the tile value regressor.  The ternary classifier's head is
 * W_h [3][w] then b_h [3]. */
int64_t nvdb_net_param_count(const nvdb_model* model, int net);

/* Copy network `net`'s flat FP32 parameters (nvdb_net_param_count floats, storage order
 * as for nvdb_mlp_grad) to / from DEVICE memory.  Stream-ordered, no synchronisation.
 * Setting them (training the networks with an optimiser of the caller's, Section 3.2)
 * repacks the tensor-core weight tiles and drops the model's patch sets and its query
 * topology, which belonged to the old weights: until nvdb_model_repatch, decompress
 * and query return NVDB_ERR_UNSUPPORTED; mlp_eval and mlp_grad work. */
nvdb_status nvdb_net_params(const nvdb_model* model, int net, float* d_out, nvdb_stream stream);
nvdb_status nvdb_net_set_params(nvdb_model* model, int net, const float* d_in, nvdb_stream stream);

/* Recompute the patch sets (Section 3.3.2) of the model's current networks against the
 * grid it encodes (same node counts, voxel count and domain; else INVALID_ARG): one set
 * per bit of patch_precs, as nvdb_compress does.  Synchronises the stream. */
nvdb_status nvdb_model_repatch(nvdb_model* model, const nvdb_grid* grid, uint32_t patch_precs, nvdb_stream stream);

nvdb_status nvdb_model_info(const nvdb_model* model, nvdb_info* out);

/* Serialise a model to a HOST buffer (format "NVDBMDL1", described below).
 * With buf == NULL, *bytes receives the size.  Synchronises the device. */
nvdb_status nvdb_model_export(const nvdb_model* model, void* buf, size_t* bytes);

/* Create a model from a HOST blob.  Errors: CORRUPT, UNSUPPORTED.
 * Synchronises the stream. */
nvdb_status nvdb_model_import(const void* buf, size_t bytes, nvdb_stream stream, nvdb_model** out);

nvdb_status nvdb_model_free(nvdb_model* model);

/* Message of the last error of the calling thread ("" if none). */
const char* nvdb_last_error(void);

/* Fault injection for tests of the failure handling; nothing here faults the GPU.
 *  NVDB_INJECT_WAIT_TIMEOUT: value != 0 makes every bounded device-side wait (the MMA
 *    completion mbarriers, the training weight staging) report a timeout once its phase
 *    has completed: the kernels take their timeout path with nothing in flight, and the
 *    calls return NVDB_ERR_TIMEOUT; value 0 clears it.
 *  NVDB_INJECT_ALLOC_BUDGET: value > 0 lets later device allocations of the library take
 *    at most `value` bytes in total, after which they fail with NVDB_ERR_OUT_OF_MEMORY
 *    (frees do not refund); value 0 removes the budget.
 *  NVDB_INJECT_STATIC_LIMIT: value in (0, 2^20] makes nvdb_mlp_grad_static use only the
 *    first `value` floats of its static array (so its capacity error can be reached with
 *    the supported network shapes); value 0 restores the full array.
 *  NVDB_INJECT_FUSED_ADAM: value 1 makes the BF16 training step apply Adam in its own
 *    (cooperative) launch after a grid-wide barrier instead of a second reduction kernel (the
 *    same result bits, measured slower); 0 the two-launch step; -1 the default (the
 *    environment variable NVDB_FUSED_ADAM=1 selects the fused step).
 * Process-wide; not for production use. */
enum { NVDB_INJECT_WAIT_TIMEOUT = 1, NVDB_INJECT_ALLOC_BUDGET = 2, NVDB_INJECT_STATIC_LIMIT = 3,
       NVDB_INJECT_FUSED_ADAM = 4 };
nvdb_status nvdb_debug_inject(int what, int64_t value);

/* Self-test of the bounded wait: one kernel waits on an mbarrier phase that nothing
 * completes, for limit_ns (at most 1 s), then returns NVDB_ERR_TIMEOUT; the device
 * stays usable.  Synchronises the device. */
nvdb_status nvdb_debug_wait_selftest(int64_t limit_ns);

/* Tracing (a measurement aid; the paper reports wall-clock times only).
 * With profiling on, the library records a CUDA event pair on the launching
 * stream around each of its kernel launches.  nvdb_profile_read waits for
 * the recorded events, aggregates them per kernel name and clears them:
 * names (HOST, cap slots of name_len chars, NUL-terminated), launches[i],
 * ms[i] (summed event time).  Returns the number of distinct names (may
 * exceed cap).  nvdb_launch_count returns the number of kernel launches the
 * library has issued since it was loaded (profiling on or off). */
void nvdb_profile_enable(int on);
int nvdb_profile_read(char* names, int name_len, int64_t* launches, double* ms, int cap);
int64_t nvdb_launch_count(void);

/*
 * Model blob "NVDBMDL1" (little-endian; every array starts at an 8-byte
 * aligned offset from the blob start; padding bytes are zero):
 *   header, 128 bytes:
 *     0 char[8] magic | 8 u32 version=1 | 12 u32 grid_class | 16 f32 background
 *     20 f32 half_width | 24 i32[3] origin | 36 i32 log2_extent
 *     40 i32[2] ffm_size (level 1, level 0) | 48 i32[3] width | 60 i32[3] layers
 *     72 i32 n_patch_sets | 76 i32 0 | 80 i64 n_l2 | 88 i64 n_l1 | 96 i64 n_leaf
 *     104 i64 n_active | 112 u64[2] 0
 *   u32 q1[m1][3], u32 q0[m0][3]   (m = ffm_size/2; fixed-point Fourier matrix,
 *        phase of frequency f at level coordinates c: sum_d q[f][d] c_d mod 2^32)
 *   per network: f32 W_0[w][n], b_0[w], W_1[w][w], b_1[w], ..., w_h[w], b_h
 *   i32 l2_origin[n_l2][3], u64 l2_mask[n_l2][512]
 *   per patch set: i32 precision, i32 0, u32 l1_off[n_l1+1], u16 l1_idx[..],
 *                  u32 l0_off[n_leaf+1], u16 l0_idx[..]
 * Network 0 (level-1 classifier) sees leaf-index coordinates (ijk - origin) >> 3
 * with q1; networks 1 and 2 see voxel coordinates ijk - origin with q0.
 */

#ifdef __cplusplus
}
#endif
#endif /* NVDB_H */
