/*
 * bbc.h -- C ABI of the GB300 effective-block-algorithm library (libbbc).
 *
 * The library computes the isospin-symmetric octet baryon-baryon four-point
 * correlators (NBS wave functions) of Nemura, "Instructive discussion of an
 * effective block algorithm for baryon-baryon correlators" (arXiv:1510.00903):
 *
 *   C_ch(r, t) = sum_X < B1_a(X + r, t) B2_b(X, t) Jbar_{B3_a' B4_b'}(t0) >
 *
 * (Sec. 2 Eq. 2 without the spin projection; Sec. 3 for the block/FFT method;
 * Sec. 4 for the 52 channels; other charge states and the decuplet Omega
 * channels of the Sec. 4 footnote) from wall-source quark propagators of a
 * light (u = d) and a strange quark.  Per time slice the work is: baryon blocks per
 * site (Sec. 3, diagrams (i)-(vi); Appendix A aggregation), a forward 3-D FFT
 * of every block field, the q-space contraction of block pairs into channels
 * (Sec. 3 Eq. LN.pLLp.FFT), an inverse 3-D FFT and the normalisation by
 * exp((m_B1 + m_B2)(t - t0)) (Sec. 2 Eq. 2).
 *
 * Conventions (all entry points):
 *  - Every call returns a bbc_status; no C++ exception crosses the ABI.  A
 *    message describing the last failure of a context is kept per context
 *    (bbc_last_error).
 *  - Device pointers are only read or written on the context's CUDA stream,
 *    asynchronously; the caller synchronises that stream before reading
 *    results on the host.  The library never frees caller memory and never
 *    allocates device memory: all device scratch lives in a workspace the
 *    caller allocates (bbc_workspace_size / bbc_set_workspace).
 *  - Propagator layout, one time slice of one flavour: S[site][12][12]
 *    complex (interleaved re, im), site = x + L*(y + L*z), row = 3*alpha + c
 *    (sink Dirac and colour index), column = 3*alpha' + c' (wall source).
 *    Dirac representation, gamma4 = diag(1,1,-1,-1), C = gamma4 gamma2.
 *  - Output layout: out[n_channels][L^3][16] complex128, spin index
 *    s = a + 2*(b + 2*(a' + 2*b')) over the upper Dirac components
 *    (a, b, a', b' in {0, 1}), r = x + L*(y + L*z) the relative distance of
 *    B1 (at X + r) and B2 (at X) -- the xi ordering of Sec. 5.
 *  - Channel ids 0..51 follow the printed order of Sec. 4 Eqs.
 *    GeneralBB_NN .. GeneralBB_XX (row by row); ids 52..55 are the four
 *    channels the paper omits because they vanish in the isospin limit
 *    (Lambda Lambda <- Sigma0 Lambda, Sigma0 Sigma0 <- Sigma0 Lambda,
 *    Sigma0 Lambda <- Lambda Lambda, Sigma0 Lambda <- Sigma0 Sigma0);
 *    ids 56..63 are other charge states (Sec. 4 footnote), each onto itself:
 *    p p, n n, Sigma+ Sigma+, Sigma- Sigma-, Xi0 Xi0, Xi- Xi-, p Sigma+,
 *    n Sigma-.  Ids 64..153 are decuplet channels (Sec. 4 footnote: the
 *    same operator form with Gamma1 = C gamma_l, Gamma2 = 1 and a spatial
 *    vector index l), with Omega-_l = eta_l eps (s^T C gamma_l s) s and
 *    eta = (i, 1, -i) for l = x, y, z (the phase that makes the operator's
 *    tensor real, like the octet ones): Omega_l1 Omega_l2 <- Omega_l3
 *    Omega_l4 at 64 + 27 l1 + 9 l2 + 3 l3 + l4, and p Omega_l <- p Omega_l'
 *    at 145 + 3 l + l' (l = 0, 1, 2).  The output keeps the 16 spin
 *    components of the upper (or lower) Dirac indices of each channel.
 *    One context holds at most 160 channels.
 */
#ifndef BBC_H
#define BBC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bbc_ctx bbc_ctx;

typedef enum {
  BBC_OK = 0,
  BBC_EINVAL = -1,   /* bad argument (size, id, null pointer, misaligned pointer) */
  BBC_ENOMEM = -2,   /* workspace missing or too small, host allocation failure */
  BBC_ECUDA = -3,    /* a CUDA runtime call failed; message in bbc_last_error */
  BBC_ESTATE = -4,   /* call out of order (e.g. contract before build) */
  BBC_ETIMEOUT = -5, /* a bounded device wait gave up (bbc_device_status) */
  BBC_ENUMERIC = -6  /* NaN or infinity in an input or output (bbc_set_checks) */
} bbc_status;

typedef enum {
  BBC_FP64 = 0,      /* blocks, FFTs, contraction and sums in FP64 */
  BBC_MIXED_FP32 = 1, /* blocks, FFTs and block-pair products in FP32 after an exact
                         per-slice power-of-two rescaling of each propagator; the signed
                         sum over Wick diagrams in double-float arithmetic (two FP32
                         words, 48-bit significand) and the normalisation in FP64.  The
                         block pairs whose operands are whole 12 x 12 open-index blocks
                         in the trace form tr(M_A(q) M_B(-q)) (most of the work for the
                         octet channels) run on the tensor cores as one complex matrix
                         product per pair {q, -q}, G(q)[i][j] = tr(M_i(q) M_j(-q)),
                         G(-q) = G(q)^T, with every FP32 operand split into two TF32
                         words (FP32-accurate products, FP32 accumulation); the other
                         pairs run on the CUDA cores in FP32.  Channel lists without such
                         pairs, or whose rows and products do not fit one CTA's shared
                         memory, run one fused CUDA-core kernel per pair {q, -q} with
                         FP64 Wick sums (the 64 octet ids fit it, and so do the 90
                         decuplet ids), or, beyond that (e.g. all octet and decuplet
                         ids together), the products and the Wick sums as two kernels
                         through a product buffer */
  BBC_MIXED_BF16 = 2, /* trial: as BBC_MIXED_FP32, with the Fourier-space blocks rounded
                         to bfloat16 (round to nearest even) before the block-pair
                         products, which multiply and accumulate in FP32; fused kernel
                         only (EINVAL at creation for channel lists that do not fit it) */
  BBC_DF64 = 3,       /* FP64-accurate results from double-float arithmetic
                         (unevaluated sums of two FP32 values, 48-bit significand) on
                         the FP32 pipes: propagators, blocks, FFTs, block-pair products
                         and Wick sums; FP64 only to split the input and to normalise */
  BBC_MIXED_TF32 = 4  /* trial: as BBC_MIXED_FP32, with the tensor-core operands rounded
                         once to TF32 (10-bit mantissa, round to nearest) instead of
                         split into two TF32 words: a third of the tensor-core work at
                         about 1e-3 relative error of the products */
} bbc_precision;

typedef enum { BBC_C128 = 0, BBC_C64 = 1 } bbc_dtype;

/* Which two Dirac components of every external spinor index (Sec. 5):
 * BBC_UPPER = indices 0, 1 (positive-parity baryons, forward in time),
 * BBC_LOWER = indices 2, 3 (negative-parity antibaryon states, backward in
 * time).  Output spins are relabelled to 0, 1 either way. */
typedef enum { BBC_UPPER = 0, BBC_LOWER = 1 } bbc_components;

typedef enum { BBC_LIGHT = 0, BBC_STRANGE = 1 } bbc_flavour;

/* Lattice description.  L: spatial extent (2, 4, 8, 16, 24, 32 or 48); T: number of time
 * slices; t0: source time slice; m_ud, m_s: quark decay masses that fix the
 * baryon masses used by the normalisation, m_B = (3 - n_s) m_ud + n_s m_s
 * (a reading for synthetic data; the paper divides by the measured masses). */
typedef struct {
  int L;
  int T;
  int t0;
  double m_ud;
  double m_s;
} bbc_lattice;

/* Create a context for one lattice, one precision and one CUDA stream
 * (cudaStream_t passed as void*; NULL = the legacy default stream).
 * channels[n_channels]: channel ids (see above), any order, no duplicates.
 * Builds the contraction plan on the host (Sec. 3 diagram classification,
 * Appendix A block aggregation); its device tables are uploaded into the
 * workspace by bbc_set_workspace.  Errors: EINVAL (bad L, T, t0, id,
 * duplicate), ENOMEM. */
bbc_status bbc_create(bbc_ctx** ctx, const bbc_lattice* lat, bbc_precision prec,
                      const int* channels, int n_channels, void* cuda_stream);

/* As bbc_create, for the given spin components of the external spinor
 * indices (bbc_create = BBC_UPPER).  With BBC_LOWER the normalisation of
 * bbc_contract uses the backward time distance d = (t0 - t) mod T. */
bbc_status bbc_create_components(bbc_ctx** ctx, const bbc_lattice* lat, bbc_precision prec, const int* channels,
                                 int n_channels, bbc_components components, void* cuda_stream);

/* Bytes of device workspace needed to process up to `slices` time slices per
 * bbc_run call (blocks of one slice, transforms, propagator copies). */
bbc_status bbc_workspace_size(const bbc_ctx* ctx, int slices, size_t* bytes);

/* Attach caller-owned device memory (256-byte aligned) of at least
 * bbc_workspace_size(ctx, slices) bytes and upload the plan tables into it
 * (asynchronously, on the context stream).  The library uses it until the
 * next bbc_set_workspace or bbc_destroy; the caller frees it after that. */
bbc_status bbc_set_workspace(bbc_ctx* ctx, void* dev_ptr, size_t bytes, int slices);

/* Copy one time slice t of one flavour into the workspace slot `slot`
 * (0 <= slot < slices): S[L^3][12][12] of dtype; on_device != 0 means `data`
 * is a device pointer, else a host pointer (pinned memory gives an
 * asynchronous copy).  The caller keeps ownership of `data`; it must stay
 * valid until the stream has passed this call. */
bbc_status bbc_load_propagator(bbc_ctx* ctx, int flavour, int slot, int t, const void* data,
                               int dtype, int on_device);

/* Step-1 of Sec. 5 for the slices in slots [0, n_slots): every aggregated
 * baryon block at every site, then its forward 3-D FFT (Sec. 3 Eq.
 * LN.pLLp.FFT, forward transform exp(-i q.x), unnormalised). */
bbc_status bbc_build_blocks(bbc_ctx* ctx, int n_slots);

/* Step-2 of Sec. 5 for slot `slot`: the q-space contraction of all channels
 * (block-pair products summed over the open colour/spin indices, then the
 * signed sum over Wick diagrams in FP64), the inverse 3-D FFT with 1/V, and
 * (normalised != 0) the factor exp((m_B1 + m_B2) d), d = (t - t0) mod T.
 * out_dev: device pointer, [n_channels][L^3][16] complex128, written fully. */
bbc_status bbc_contract(bbc_ctx* ctx, int slot, void* out_dev, int normalised);

/* Plan statistics of one channel (position in the context's channel list)
 * and one pair of source operator terms (term3 of B3, term4 of B4; the
 * X_u, X_d, X_s terms of Lambda / Sigma0 in that order, 0 otherwise):
 * n_diagrams and, per diagram, the number of iterations of its open-index
 * sum (1, 9, 36 or 144) times the parity of its Wick permutation (+1/-1)
 * written to iters_signed[0 .. min(n, cap)).  Reproduces the paper's
 * Tables of iteration counts (Sec. 4). */
bbc_status bbc_plan_stats(const bbc_ctx* ctx, int channel_pos, int term3, int term4,
                          int* n_diagrams, int* iters_signed, int cap);

/* Aggregated plan sizes: unique blocks, block outputs per site, block-pair
 * products per q (16 spin combinations per aligned block pair) and their
 * complex multiply-adds per site. */
bbc_status bbc_plan_sizes(const bbc_ctx* ctx, int* n_blocks, int* n_block_outputs,
                          int* n_pair_items, long long* pair_macs_per_site);

/* The whole contraction plan as host tables (no device work), so that a host
 * program can evaluate the block algorithm of Sec. 3 step by step (the tests
 * do, on tiny lattices, against the oracle).  Call once with every array
 * NULL to receive sizes[5] = {n_out (block rows per site), n_terms,
 * n_tasks, n_items, n_outputs = 16 x channels}; then again with the arrays
 * (owned by the caller) and sizes[] holding their capacities in the same
 * units: the call fills them all, or, if any array is NULL, none; if a
 * capacity is too small it fills none, returns BBC_EINVAL and leaves the
 * needed sizes in sizes[]:
 *  row_ptr[n_out + 1], terms[n_terms][3]: block row r is the sum over terms
 *    row_ptr[r] .. row_ptr[r+1]-1 of weight x F_family[index], with
 *    (family, index, weight) per term; family 0..6 = (l,l,l), (l,l,s),
 *    (l,s,l), (l,s,s) with Gamma1 = C gamma5 and (s,s,s) with eta_l C
 *    gamma_l, l = x, y, z; index = a*1728 + e0*144 + e1*12 + e2 of
 *    F[a][e0][e1][e2] = sum eps(c0,c1,c2) Gamma1(a0,a1) S_f0[(a0,c0),e0]
 *    S_f1[(a1,c1),e1] S_f2[(a+o,c2),e2] (o = 0 upper, 2 lower components);
 *  tasks[n_tasks][24] = nA, nB, n1, n2, sA1, sA2, sB1, sB2, offA[8],
 *    offB[8]: P[16 t + rA nB + rB](q) = sum over i1 < n1, i2 < n2 of
 *    A[offA[rA] + i1 sA1 + i2 sA2](q) A[offB[rB] + i1 sB1 + i2 sB2](-q), A
 *    the Fourier transform (exp(-i q.x)) of the block rows;
 *  out_ptr[n_outputs + 1], items[n_items], coefs[n_items]: Ct[o](q) = sum
 *    of coefs[c] P[items[c]](q), o = 16 channel_pos + spin; the raw
 *    correlator is the inverse transform of Ct divided by V. */
bbc_status bbc_plan_export(const bbc_ctx* ctx, int* sizes, int* row_ptr, int* terms, int* tasks, int* out_ptr,
                           int* items, double* coefs);

/* Stages timed by bbc_stage_timing. */
typedef enum {
  BBC_STAGE_INGEST = 0,     /* propagator rescaling copy (per flavour and slice) */
  BBC_STAGE_BUILD = 1,      /* baryon blocks of every site */
  BBC_STAGE_FFT_FWD = 2,    /* forward 3-D FFT of every block field (3 passes) */
  BBC_STAGE_CONTRACT = 3,   /* q-space block-pair products (all spins, summed over open indices) */
  BBC_STAGE_FFT_INV = 4,    /* inverse 3-D FFT with the fused output transpose and normalisation */
  BBC_STAGE_NORMALISE = 5,  /* per-channel normalisation factors */
  BBC_STAGE_WICK = 6,       /* signed FP64 sums of pair products over Wick diagrams */
  BBC_STAGE_PROJECT = 7,    /* spin-state and cubic-group projections (bbc_project) */
  BBC_N_STAGES = 8
} bbc_stage;

/* enable != 0: from now on bracket every stage launch with CUDA events on the
 * context stream (events are created by the library; no device memory).
 * enable == 0: stop.  Either way the accumulated record is cleared. */
bbc_status bbc_enable_stage_timing(bbc_ctx* ctx, int enable);

/* Synchronise the context stream, then write per stage the summed device
 * time in milliseconds (ms[BBC_N_STAGES]) and the number of timed stage
 * launches (launches[BBC_N_STAGES], one per API call that ran the stage) since
 * timing was enabled or last read; clears the record. */
bbc_status bbc_stage_timing(bbc_ctx* ctx, double* ms, long long* launches);

/* Number of kernel launches one bbc_contract call issues, and one
 * bbc_build_blocks call per slot-batch, and one bbc_load_propagator call. */
bbc_status bbc_launch_counts(const bbc_ctx* ctx, int* per_load, int* per_build, int* per_contract);

/* One item of a batch: a time slice of one context. */
typedef struct {
  bbc_ctx* ctx;            /* its lattice, precision, channels and workspace */
  int t;                   /* time slice, 0 <= t < T of the context */
  const void* S_light;     /* [L^3][12][12] propagators of dtype (as bbc_load_propagator) */
  const void* S_strange;
  int dtype;               /* BBC_C128 or BBC_C64 */
  int on_device;           /* 1: device pointers; 0: host memory (pinned for asynchronous copies) */
  void* out_dev;           /* [n_channels][L^3][16] complex128 (device) */
  int normalised;
} bbc_batch_item;

/* Batch entry point (many slices, sources, gauge samples and uneven
 * lattices in one call): runs items[0 .. n_items) in order on cuda_stream.
 * Consecutive items of one context form waves of up to its slot count
 * (bbc_set_workspace's slices): the propagators of the wave's items go into
 * slots 0 .. k-1, one block build and one forward FFT run over the k slots
 * (in the mixed precisions at L <= 32 the FFT is one queue-driven launch over
 * every row tile of the k slices), then the k contractions write each item's
 * out_dev.  Every launch and copy is on cuda_stream (the contexts' own
 * streams are not used; they are restored before returning).  Capturing
 * cuda_stream into a CUDA graph around this call records the whole batch as
 * one graph.  Contexts may share a workspace (their work is ordered on the
 * one stream).  Asynchronous unless a context has numeric checks on.
 * Errors: the status of the first failing call; *failed_item (if not NULL)
 * gets the item whose load or contraction failed, or the first item of the
 * wave whose build failed (a batch resumes from there); EINVAL for a null or
 * empty batch. */
bbc_status bbc_batch_run(const bbc_batch_item* items, int n_items, void* cuda_stream, int* failed_item);

/* Numeric checks (off by default).  BBC_CHECK_INPUT: bbc_load_propagator
 * returns BBC_ENUMERIC when the slice has a NaN or infinite entry.
 * BBC_CHECK_OUTPUT: bbc_contract returns BBC_ENUMERIC when a correlator it
 * wrote is NaN or infinite.  Each check synchronises the context stream (not
 * inside a stream capture). */
#define BBC_CHECK_INPUT 1
#define BBC_CHECK_OUTPUT 2
bbc_status bbc_set_checks(bbc_ctx* ctx, int flags);

/* Bounded device waits.  In the mixed precisions (L <= 32) the forward 3-D FFT
 * of bbc_build_blocks is one persistent launch whose CTAs take (row tile,
 * z plane) and (row tile, z lines) units from a device work queue; a z-lines
 * unit waits for the planes of its row tile, at most about a second, and a
 * wait that gives up sets a sticky device word and stops the launch.  The
 * tensor-core contraction of the mixed precisions (one persistent CTA per SM,
 * tcgen05 products committed to mbarriers) bounds its mbarrier waits the
 * same way and sets another bit of the word.  bbc_device_status synchronises
 * the context stream and returns BBC_ETIMEOUT if either happened since the
 * last call (the word is cleared; after an FFT timeout every slot is marked
 * unbuilt, its blocks not being valid; after a contraction timeout the
 * correlators of that contraction are not valid), else BBC_OK (also without a
 * workspace).  BBC_CHECK_OUTPUT runs the same check in bbc_contract.  Not
 * inside a stream capture. */
bbc_status bbc_device_status(bbc_ctx* ctx);

/* Self-test of those waits: one queue-driven forward FFT of slot 0's blocks
 * with a dependency count no unit reaches, so that every wait runs out after
 * spin_limit polls (1 .. 2^22, each about 0.3 us).  Synchronous.  Returns
 * BBC_ETIMEOUT when the kernel reported the timeout (the expected outcome;
 * slot 0 is then unbuilt and the context usable), BBC_OK if no wait gave up
 * (a fault in the waits), EINVAL for spin_limit out of range, ESTATE without a
 * workspace or without the queue-driven FFT (FP64, double-float, L = 48, or
 * a plan too large for the fused kernels).  Not inside a stream capture. */
bbc_status bbc_check_bounded_wait(bbc_ctx* ctx, long long spin_limit);

/* Launch configuration of the two kernels whose shape is tunable:
 *  build_sites, build_threads: sites per CTA and threads of the block build,
 *    one of (1, 256), (2, 256), (2, 512), (4, 512), (1, 512); a CTA keeps the
 *    propagators, diquarks and sink-tensor entries of its sites in shared
 *    memory (configurations that need more than 227 KB are not valid);
 *  fused_warps, fused_chunk (mixed precisions with the fused kernel only): warps per CTA (8, 12, 16)
 *    of the fused q-space contraction and the open-index steps per warp unit
 *    (18, 36, 72, 144), or 0: each warp takes one contiguous run of the
 *    batches' steps of equal modelled cost;
 *  fused_steps: open-index steps whose rows a lane loads before multiplying
 *    (1; or 2 with 8 or 12 warps, which leave the registers for it);
 *  pair_groups (BBC_FP64, BBC_DF64 and the unfused FP32 route): warp task
 *    lists of the block-pair products per 32 q (48, 96, 192 or 384); more,
 *    shorter lists shorten the tail of the launch;
 *  tc_kernel (mixed FP32 / TF32 with tensor cores): 0 = the trace-form
 *    products on tcgen05 (one persistent CTA per SM, then the CUDA-core
 *    kernel), 1 = on mma.sync, with the CUDA-core kernel of one quarter of
 *    the pairs beside the tensor-core kernel of the next on a second stream
 *    from 4096 pairs {q, -q} on.
 * A new context starts with (1, 256, 16, 18, 1, 48, 0) (pair_groups 192 for
 * BBC_DF64), or with the configuration bbc_autotune chose earlier in the
 * process for the same L, precision and channel list. */
typedef struct {
  int build_sites, build_threads;
  int fused_warps, fused_chunk, fused_steps;
  int pair_groups;
  int tc_kernel;
} bbc_tuning;

bbc_status bbc_get_tuning(const bbc_ctx* ctx, bbc_tuning* out);

/* Set a configuration (EINVAL if unsupported; the fused fields are ignored
 * without the fused kernel, pair_groups with it).  Synchronises the context
 * stream when a workspace is attached (uploads the warp schedule).  Not
 * inside a stream capture. */
bbc_status bbc_set_tuning(bbc_ctx* ctx, const bbc_tuning* t);

/* Autotuner: times every valid candidate configuration with CUDA events on
 * the context stream, `reps` launches each after one untimed launch, on the
 * propagators loaded in slot 0 -- the block-build candidates in the order
 * above, then (fused kernel) every valid (fused_warps, fused_steps,
 * fused_chunk) in row-major order (warps 8, 12, 16; steps 1, 2; chunks 0, 18,
 * 36, 72, 144) and then, with tensor cores, tc_kernel 0 and 1, or
 * (otherwise) pair_groups 48, 96, 192, 384 for the block-pair products --
 * keeps the fastest of each kernel, rebuilds slot 0 with
 * it, and records it for later contexts with the same L, precision and
 * channel list.  ms[i] (i < cap) receives the average milliseconds per launch
 * of candidate i (-1 for a candidate that is not valid here); *n_tried the
 * number of candidates; *best the chosen configuration.  ms, best, n_tried
 * may be NULL.  Synchronous; not inside a stream capture.  Errors: ESTATE (no
 * workspace, slot 0 not loaded), EINVAL (reps outside [1, 1000]), ECUDA. */
bbc_status bbc_autotune(bbc_ctx* ctx, int reps, bbc_tuning* best, double* ms, int cap, int* n_tried);

/* Projections of Sec. 2 (the source operator of total spin J, M in the
 * equation for R^(J,M), and the operator P of the 3S1 / 3D1 split) applied to
 * correlators in the layout bbc_contract writes: C_dev[n_fields][L^3][16]
 * complex128, spin s = a + 2(b + 2(a' + 2 b')), index 0 = spin up.
 *
 *   R[f][r][a + 2b + 4 jm]  = sum_{a'b'} P^(J,M)_{a'b'} C[f][r][a + 2b + 4a' + 8b']
 *   Ra1[f][r][j]            = (1/24) sum over the 24 rotations g of the cube of R[f][g r][j]
 *
 * States jm = 0: (J,M) = (0,0) = (|ud> - |du>)/sqrt2, 1: (1,+1) = |uu>,
 * 2: (1,0) = (|ud> + |du>)/sqrt2, 3: (1,-1) = |dd> (Clebsch-Gordan
 * coefficients, Condon-Shortley phases); the rotations act on the relative
 * coordinate r on the periodic lattice, the sink spins a, b are untouched.
 * The D-wave part of Sec. 2 is R - Ra1.  R_dev or Ra1_dev may be NULL (not
 * both); neither may overlap C_dev.  All three are device pointers, 16-byte
 * aligned, of n_fields * L^3 * 16 complex128 (L of the context).  FP64 on the
 * context stream, asynchronous; needs the workspace attached (it holds the
 * orbit table of the rotations on the lattice).  Errors: EINVAL, ESTATE. */
bbc_status bbc_project(bbc_ctx* ctx, const void* C_dev, int n_fields, void* R_dev, void* Ra1_dev);

/* Bytes of the static device array used by bbc_run_slice_static. */
#define BBC_STATIC_SCRATCH_BYTES (32u * 1024u * 1024u)

/* One time slice of the whole path without any device allocation, for
 * callers that cannot call cudaMalloc (a process whose device memory belongs
 * to another runtime's pool allocator, a plugin inside such a process, or a
 * loop that must not take an allocation's implicit synchronisation).  The
 * paper has no counterpart: it is an interface for such callers.
 *
 * Computes what bbc_load_propagator (both flavours, one slot), bbc_build_blocks
 * and bbc_contract compute for time slice t, with every byte of device scratch
 * in one file-scope __device__ array of BBC_STATIC_SCRATCH_BYTES (32 MiB)
 * that every GPU loading the library holds from module load until exit.  No
 * workspace needs to be attached.  S_light, S_strange: device pointers,
 * [L^3][12][12] of dtype (16-byte aligned); out_dev: device pointer,
 * [n_channels][L^3][16] complex128, written fully.  Everything runs
 * asynchronously on the context stream.
 *
 * Precisions BBC_FP64 and BBC_MIXED_FP32 (EINVAL for the others); the
 * contraction runs on the CUDA cores (block-pair products, then Wick sums)
 * whatever the context's precision would pick otherwise.  Contexts with
 * numeric checks (bbc_set_checks) are rejected with EINVAL.
 * Size limit: the plan tables and one slice of blocks, pair products and
 * q-space correlators must fit in the array -- L <= 4 with all 52 channels;
 * larger lattices or channel lists return BBC_EINVAL with a message.
 * Every call copies the plan tables from host memory into the array.  The
 * first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current, and the first call with a
 * context uploads the FFT twiddle tables (synchronously); make that first
 * call before any stream capture.  All calls share the one array and leave
 * their data in it: calls whose work overlaps on the GPU (other streams,
 * other host threads without ordering) race on it.  Allocates no device
 * memory; host memory only for the error message of a failed call. */
bbc_status bbc_run_slice_static(bbc_ctx* ctx, int t, const void* S_light, const void* S_strange, int dtype,
                                void* out_dev, int normalised);

/* Message of the last failed call on ctx (or of the last failed bbc_create
 * when ctx is NULL).  Valid until the next call on the same context. */
const char* bbc_last_error(const bbc_ctx* ctx);

/* Release the context and its plan tables (not the caller's workspace). */
void bbc_destroy(bbc_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* BBC_H */
