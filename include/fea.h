/*
 * fea.h -- C ABI of the GB300 finite-element assembly library.
 *
 * The library assembles convection-diffusion-reaction (CDR) transport equations
 * (species mass fractions, enthalpy) element by element on an unstructured mesh
 * into one shared CSR pattern, on one GPU.  The paper it follows is
 * "Performance assessment of CUDA and OpenACC in large scale combustion
 * simulations" (arXiv 2107.11541):
 *   - Sec. 4.2, Listing 1: the element loop (outer loop over elements, inner
 *     loop over Gauss points and node pairs building the element matrix Ae from
 *     shape functions N and the Jacobian weight Jac(g) = w_g det J_g);
 *   - Sec. 4.2: the assembled matrix is stored in CSR;
 *   - Sec. 2 and Table 1: heat and species equations, whose matrix assembly is
 *     most of the time step;
 *   - Sec. 4.3, Fig. 3: elements grouped by type and packed in fixed-size
 *     packs with zero padding (see fea_pack_plan).
 * The paper does not write the transport equations.  The operator assembled is
 * the backward-Euler Galerkin + SUPG discretisation of
 *     d(phi)/dt + u.grad(phi) - div(k grad(phi)) + s phi = 0,
 * per Gauss point g with dV = w_g det J_g:
 *     A_ab += dV [ N_a N_b/dt + N_a u.grad N_b + k grad N_a.grad N_b + s N_a N_b
 *                  + tau (u.grad N_a)(N_b/dt + u.grad N_b + s N_b) ]
 *     b_a  += dV (N_a + tau u.grad N_a) phi_old / dt
 * with u, k, s, phi_old interpolated from nodal values, tau = 1/(4k/h^2 + 2|u|/h + s)
 * (0 if the denominator is 0) and h = V_e^(1/3)/p.
 *
 * Conventions common to every call
 *   - All calls return fea_status and never abort or trap.  On failure
 *     fea_last_error() returns a thread-local message.
 *   - Node ids are 0-based int32.  Local node order: Tet4 positively oriented
 *     ((x1-x0)x(x2-x0).(x3-x0) > 0); Hex8 a = i + 2j + 4k and Hex27
 *     a = i + 3j + 9k, with i, j, k the node's position along xi, eta, zeta;
 *     Pen6 (prism) nodes 0-2 a triangle and 3-5 the opposite triangle, node
 *     a + 3 across from node a, with (x1-x0)x(x2-x0).(x3-x0) > 0; Pyr5
 *     (pyramid) nodes 0-3 the base quad counter-clockwise seen from the apex,
 *     node 4 the apex.
 *   - Element types and Gauss rules (Sec. 2 and Sec. 4.2: unstructured meshes
 *     mixing tetrahedra, prisms, pyramids and hexahedra; the paper gives no
 *     rules): Tet4 4 points (degree 2); Hex8 2x2x2 and Hex27 3x3x3 Gauss;
 *     Pen6 linear triangle x linear line, 3 x 2 points; Pyr5 rational base
 *     functions (1/4)[(1-z) + xa x + ya y + xa ya x y/(1-z)] and apex z on the
 *     reference pyramid |x|,|y| <= 1-z, 0 <= z <= 1, 2x2x3 points of a cube
 *     collapsed onto it.  h = V_e^(1/3) / p with p = 2 for Hex27, else 1.
 *   - Device work is ordered on the mesh's CUDA stream.  Calls that only
 *     enqueue work return without waiting; device-detected errors are
 *     reported by the next call that waits (fea_sync, fea_pattern_build,
 *     fea_mesh_create) as FEA_ERR_* codes.
 *   - Array layouts are row-major C arrays; "[a][b]" means b is fastest.
 */
#ifndef FEA_H
#define FEA_H

#include <stdint.h>

#if defined(__GNUC__)
#define FEA_API __attribute__((visibility("default")))
#else
#define FEA_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fea_mesh fea_mesh;
typedef struct fea_pattern fea_pattern;
typedef struct fea_graph fea_graph;

typedef enum { FEA_TET4 = 0, FEA_HEX8 = 1, FEA_HEX27 = 2, FEA_PEN6 = 3, FEA_PYR5 = 4 } fea_elem_t;

typedef enum {
  FEA_OK = 0,
  FEA_ERR_ARG = 1,        /* bad argument: null pointer, negative size, unknown enum, n_eq <= 0, dt <= 0 */
  FEA_ERR_RANGE = 2,      /* a connectivity entry is outside [0, n_node) */
  FEA_ERR_DUP_NODE = 3,   /* a node appears twice in one element */
  FEA_ERR_INVERTED = 4,   /* det J <= 0 at a Gauss point or a corner of an element */
  FEA_ERR_TOO_LARGE = 5,  /* a size exceeds an index type: nnz >= 2^31, n_node >= 2^31, or a row too long */
  FEA_ERR_OOM = 6,        /* device or host allocation failed */
  FEA_ERR_CUDA = 7,       /* a CUDA runtime call failed */
  FEA_ERR_TIMEOUT = 8,    /* a bounded device-side wait gave up */
  FEA_ERR_STATE = 9       /* object used in the wrong state (e.g. pattern of another mesh) */
} fea_status;

typedef enum {
  FEA_F64_PLAIN = 0,  /* double fields and outputs; one launch per equation, geometry recomputed each time */
  FEA_F32_FUSED = 1   /* float fields and outputs; all equations in one launch sharing the geometry */
} fea_precision;

enum {
  FEA_TERM_MASS = 1,  /* N_a N_b / dt, and the Galerkin RHS N_a phi_old / dt */
  FEA_TERM_CONV = 2,  /* N_a u.grad N_b */
  FEA_TERM_DIFF = 4,  /* k grad N_a . grad N_b */
  FEA_TERM_REAC = 8,  /* s N_a N_b */
  FEA_TERM_SUPG = 16, /* tau (u.grad N_a)(N_b/dt + u.grad N_b + s N_b), and its RHS part */
  FEA_TERM_ALL = 31
};

typedef enum {
  FEA_SCATTER_AUTO = 0,     /* autotuned: the first FP32 call for a pattern, equation count and term mask
                               times the candidates of fea_tune_candidates (scatter x equation groups x
                               Gauss-point mapping x elements per CTA x Hex27 contraction; those too
                               large to try are skipped; row-owned batch sizes are tried for the best
                               group count only) and keeps the fastest; the choice is also stored in and
                               read back from the tuning cache file (see fea_tuned_config).  Not tuned
                               while the stream is capturing or with accumulate = 1: then row-owned if
                               available, else atomic, with the type kernels */
  FEA_SCATTER_ATOMIC = 1,   /* element-parallel, atomic adds into zeroed outputs */
  FEA_SCATTER_ROWOWNED = 2, /* rows accumulated in shared memory and written once (deterministic) */
  FEA_SCATTER_GATHER = 3    /* FP32 only: element matrices to a device scratch buffer owned by the pattern,
                               then every CSR row summed by one warp over its incident elements in
                               ascending element order and written once (deterministic) */
} fea_scatter;

typedef enum {
  FEA_CONTRACT_AUTO = 0,      /* autotuned with the scatter (see FEA_SCATTER_AUTO); CUDA cores when not tuned */
  FEA_CONTRACT_CUDA = 1,      /* FP32 products on the CUDA cores */
  FEA_CONTRACT_TC_BF16X3 = 2, /* tensor cores: each operand split into two BF16 parts, products
                                 hi hi + hi lo + lo hi (about 16 bits of each operand), FP32 accumulation */
  FEA_CONTRACT_TC_TF32X3 = 3  /* tensor cores: two TF32 parts (the value with its 13 low mantissa bits
                                 cleared, and the exact remainder), the same three products (about 22
                                 bits of each operand), FP32 accumulation */
} fea_contraction;

typedef enum {
  FEA_MAP_AUTO = 0,             /* autotuned with the scatter (see FEA_SCATTER_AUTO); else FEA_MAP_TYPE_KERNEL */
  FEA_MAP_TYPE_KERNEL = 1,      /* the kernel specialised for the element type: one thread per (element,
                                   equation) walking the Gauss points (Tet4, Pen6, Pyr5; batched for Hex8,
                                   with one thread per (element, Gauss point) for the shared geometry), or one
                                   CTA per element with threads over (Gauss point, node) tasks (Hex27) */
  FEA_MAP_WARP_PER_ELEMENT = 2, /* one warp per element, any type: lanes over the Gauss points for the
                                   geometry, then over the matrix entries */
  FEA_MAP_TWO_THREADS_PER_ITEM = 3 /* row-owned Hex8 scatter, full operator: two threads per (element,
                                   equation), each forming four rows of the element matrix, in CTAs of 512
                                   threads (twice the warps per SM); elsewhere as FEA_MAP_TYPE_KERNEL */
} fea_mapping;

typedef struct {
  int32_t precision;        /* fea_precision, default FEA_F32_FUSED */
  int32_t terms;            /* bit mask of FEA_TERM_*, default FEA_TERM_ALL */
  int32_t scatter;          /* fea_scatter, default FEA_SCATTER_AUTO */
  int32_t accumulate;       /* 0: overwrite values/rhs (default); 1: add to them */
  double kappa_threshold;   /* F32 path: Gauss points whose Jacobian condition estimate |J|_F |J^-1|_F (an
                               upper bound of the 2-norm condition number, 3 for a scaled identity)
                               exceeds this get FP64 geometry (default 1e3) */
  void* event_begin;        /* optional cudaEvent_t recorded on the mesh stream just before the assembly
                               kernel(s), after any output zeroing; NULL = none */
  void* event_end;          /* optional cudaEvent_t recorded just after the assembly kernel(s) */
  int32_t eq_groups;        /* row-owned scatter: equations are assembled in this many groups (geometry
                               recomputed per group, more rows per shared-memory window); 0 = 1, or the
                               autotuned count under FEA_SCATTER_AUTO */
  int32_t cancel_check;     /* FP32 path: 1 = rows whose sums cancel are redone in FP64 (see
                               fea_cancel_rows); not allowed with accumulate.  Default 0 */
  int32_t host_parts;       /* fea_assemble_host only: the equations are assembled in this many parts,
                               each part's inputs copied in and values copied back while other parts
                               compute (at most n_eq); 0 = automatic: when the values exceed 256 MB and
                               n_eq >= 3, about 16 GB of values per part and at least 3 parts, else 1.
                               Default 0 */
  int32_t contraction;      /* fea_contraction: how the FP32 Hex27 element matrices (full operator, up to
                               12 equations) are contracted; other element types and the residual use
                               the CUDA cores.  Default FEA_CONTRACT_AUTO */
  int32_t mapping;          /* fea_mapping: Gauss-point-to-thread mapping of the FP32 element kernels
                               (atomic and gather scatters, residual).  Default FEA_MAP_AUTO */
  int32_t elems_per_cta;    /* FP32 work per CTA, 0 = the kernel's own rule (default): elements per batch
                               of the Hex8 kernels (row-owned: 1-32, element-parallel: 1-96); threads per
                               CTA, one (element, equation) each, of the Tet4 (128 or 256) and Pen6/Pyr5
                               (64 or 128) kernels; ignored elsewhere */
  int32_t reserved[2];
} fea_assemble_opts;

/* One autotuned configuration (fea_tuned_config, fea_tune_candidates). */
typedef struct {
  int32_t scatter;          /* fea_scatter */
  int32_t eq_groups;        /* equation groups (row-owned scatter), else 1 */
  int32_t mapping;          /* fea_mapping */
  int32_t elems_per_cta;    /* 0 = the kernel's rule */
  int32_t contraction;      /* fea_contraction */
  int32_t from_cache;       /* 1 when taken from the tuning cache file instead of timed in this process */
  float ms;                 /* the timed assembly, ms (as recorded in the cache when from_cache = 1) */
} fea_tuning;

/* Fills *opts with the defaults listed above. */
FEA_API fea_status fea_default_opts(fea_assemble_opts* opts);

/*
 * fea_mesh_create -- copy a mesh to the device and validate it.
 *   coords  [n_node][3] double, host or device pointer (detected), copied.
 *   conn    [n_elem][nen] int32, host or device pointer (detected), copied.
 *   stream  cudaStream_t used for all work on this mesh (NULL = legacy default stream).
 *   *out    receives the mesh, owned by the caller, released with fea_mesh_destroy.
 * Checks (on the device, writing a status word; never traps): ids in range
 * (FEA_ERR_RANGE), no repeated node in an element (FEA_ERR_DUP_NODE), det J > 0
 * at every Gauss point and corner (FEA_ERR_INVERTED).  Waits for the stream.
 * n_elem = 0 is allowed (an empty mesh assembles to the mass-free zero matrix).
 */
FEA_API fea_status fea_mesh_create(const double* coords, int64_t n_node, const int32_t* conn, int64_t n_elem,
                           fea_elem_t type, void* stream, fea_mesh** out);

/*
 * fea_mesh_create_mixed -- a mesh of n_blocks element blocks of different types sharing
 * one node set (Sec. 2 and Sec. 4.2: one unstructured mesh of several element kinds;
 * elements grouped by type as in Sec. 4.3).
 *   coords       [n_node][3] double, host or device pointer, copied.
 *   types[b]     element type of block b (host array of n_blocks).
 *   conns[b]     [n_elems[b]][nen of types[b]] int32, host or device pointer, copied
 *                (host array of n_blocks pointers; may be NULL where n_elems[b] = 0).
 *   n_elems[b]   elements of block b (host array).
 * Elements are numbered block by block.  Validation as in fea_mesh_create, per block.
 * n_blocks = 1 gives the single-type mesh of fea_mesh_create.  On a mesh of several
 * types the position map of fea_pattern_get holds block b's [n_elems[b]][nen_b][nen_b]
 * array after those of blocks 0..b-1; fea_assemble scatters with atomics (AUTO or
 * ATOMIC; ROWOWNED, GATHER and the cancellation check return FEA_ERR_ARG); fea_residual,
 * fea_assemble_host, fea_spmv and the step graph work as on any mesh.
 */
FEA_API fea_status fea_mesh_create_mixed(const double* coords, int64_t n_node, int32_t n_blocks,
                                         const fea_elem_t* types, const int32_t* const* conns,
                                         const int64_t* n_elems, void* stream, fea_mesh** out);
FEA_API fea_status fea_mesh_destroy(fea_mesh* mesh);
/* Rebinds the mesh (and its patterns) to another stream. */
FEA_API fea_status fea_mesh_set_stream(fea_mesh* mesh, void* stream);
/* Waits for the mesh's stream and returns any error the device recorded. */
FEA_API fea_status fea_sync(fea_mesh* mesh);

/*
 * fea_pattern_build -- the CSR sparsity pattern of the mesh (Sec. 4.2: CSR storage).
 * Row i holds column j iff some element contains both nodes i and j (j = i
 * included); columns ascend.  Also builds the position map
 * pos[e][a][b] = the index k in row conn[e][a] with colind[k] = conn[e][b], and
 * the internal schedules the assembly kernels use.  All results stay on the
 * device and are owned by the pattern.  Fails with FEA_ERR_TOO_LARGE when
 * nnz >= 2^31.  Waits for the stream.
 */
FEA_API fea_status fea_pattern_build(fea_mesh* mesh, fea_pattern** out);
/* Borrowed device pointers: rowptr int64[n_node+1], colind int32[nnz], pos int32[n_elem][nen][nen]
 * (on a mesh of several types: every block's array in turn, see fea_mesh_create_mixed). */
FEA_API fea_status fea_pattern_get(const fea_pattern* pattern, const int64_t** rowptr, const int32_t** colind,
                           const int32_t** pos, int64_t* nnz);
FEA_API fea_status fea_pattern_destroy(fea_pattern* pattern);

/*
 * fea_assemble -- assemble n_eq CDR equations sharing one mesh and pattern.
 * All array arguments are DEVICE pointers owned by the caller, of element type
 * double for FEA_F64_PLAIN and float for FEA_F32_FUSED:
 *   velocity    [3][n_node]     nodal velocity, shared by all equations (SoA)
 *   diffusivity [n_eq][n_node]  nodal k per equation
 *   reaction    [n_eq][n_node]  nodal s per equation
 *   phi_old     [n_eq][n_node]  previous-step nodal values per equation
 *   values      [n_eq][nnz]     output: CSR values, one standalone matrix per equation
 *   rhs         [n_eq][n_node]  output: right-hand sides
 * dt > 0 is the time step; opts may be NULL for the defaults.  Enqueued on the
 * mesh's stream; returns without waiting.
 */
FEA_API fea_status fea_assemble(fea_mesh* mesh, const fea_pattern* pattern, const void* velocity,
                        const void* diffusivity, const void* reaction, const void* phi_old, double dt,
                        int32_t n_eq, const fea_assemble_opts* opts, void* values, void* rhs);

/*
 * fea_residual -- the matrix-free residual of the same discretisation at a field phi:
 *     r[q][n] = b_q[n] - sum_e (A^e_q phi^e_q)[n]
 * formed element by element without building the CSR matrix (an explicit step applies the
 * operator rather than solving with it, Sec. 2).  A^e and b^e are exactly the element
 * contributions fea_assemble sums, so r = rhs - values * phi up to rounding.
 *   velocity, diffusivity, reaction, phi_old: as in fea_assemble
 *   phi  [n_eq][n_node] the field the operator is applied to
 *   r    [n_eq][n_node] output (opts->accumulate = 1 adds to it)
 * Precision and term mask from opts; the scatter option is ignored (atomic adds into the
 * zeroed r).  Device arrays, enqueued on the mesh's stream.
 */
FEA_API fea_status fea_residual(fea_mesh* mesh, const fea_pattern* pattern, const void* velocity,
                                const void* diffusivity, const void* reaction, const void* phi_old, const void* phi,
                                double dt, int32_t n_eq, const fea_assemble_opts* opts, void* r);

/*
 * fea_explicit_step -- one explicit time step of every equation (Sec. 2: heat and species
 * advance by a third-order Runge-Kutta scheme without an algebraic solver):
 *     M_L dphi/dt = -A phi,
 * A the convection, diffusion and reaction terms of the operator (those selected by opts->terms
 * among FEA_TERM_CONV, FEA_TERM_DIFF, FEA_TERM_REAC; the mass and SUPG bits are ignored), applied
 * element by element as in fea_residual, and M_L[i] = sum_j M_ij = int N_i dV the row-sum lumped
 * mass.  stages = 1: forward Euler phi += dt L(phi); stages = 3: the strong-stability-preserving
 * RK3 scheme phi1 = phi + dt L(phi), phi2 = 3/4 phi + 1/4 (phi1 + dt L(phi1)),
 * phi = 1/3 phi + 2/3 (phi2 + dt L(phi2)), with L(x) = -M_L^-1 A x.
 *   velocity, diffusivity, reaction: as in fea_assemble (DEVICE arrays of the precision in opts)
 *   phi  [n_eq][n_node] DEVICE array: the field, advanced in place
 *   dt   > 0; keeping it within the explicit stability limit is the caller's part
 * The lumped mass is computed by the first call for a pattern and precision (it waits for the
 * stream once) and kept; the stage buffers (3 n_eq n_node values) are a device workspace owned
 * by the pattern, grown on demand.  Enqueued on the mesh's stream; opts->event_begin/event_end
 * bracket the step.  FEA_ERR_ARG for stages other than 1 or 3, or a term mask with none of the
 * three terms.
 */
FEA_API fea_status fea_explicit_step(fea_mesh* mesh, const fea_pattern* pattern, const void* velocity,
                                     const void* diffusivity, const void* reaction, void* phi, double dt,
                                     int32_t n_eq, int32_t stages, const fea_assemble_opts* opts);

/*
 * fea_assemble_host -- the same operation on HOST arrays (same shapes and
 * types as fea_assemble).  Copies the inputs to a device workspace owned by the
 * pattern, assembles, copies values and rhs back, and waits for completion.  With
 * several parts (opts->host_parts) each part's field slices are copied in on their own
 * streams ahead of its assembly and its values copied back while later parts compute.
 * Pinned host memory gives the fastest copies.
 */
FEA_API fea_status fea_assemble_host(fea_mesh* mesh, const fea_pattern* pattern, const void* velocity,
                             const void* diffusivity, const void* reaction, const void* phi_old, double dt,
                             int32_t n_eq, const fea_assemble_opts* opts, void* values, void* rhs);

/*
 * fea_pack_plan -- the element-pack layout of Sec. 4.3 / Fig. 3: elements of
 * each type are grouped, then cut into packs of vector_size elements, the last
 * pack zero-padded.  For n_types counts, writes packs[t] and pads[t].  Host only.
 */
FEA_API fea_status fea_pack_plan(const int64_t* count_by_type, int32_t n_types, int32_t vector_size, int64_t* packs,
                         int64_t* pads);

/*
 * fea_csr_rowptr_noalloc -- CSR row pointers from per-row counts, allocating nothing.
 * The paper has no counterpart.  It is the row-pointer step of fea_pattern_build, offered
 * to callers that cannot let a library allocate device memory: for example a program whose
 * device memory all belongs to its own pool or arena.
 *   counts  [n] int32 DEVICE pointer, caller-owned: counts[i] >= 0 columns in row i
 *   rowptr  [n+1] int64 DEVICE pointer, caller-owned output:
 *           rowptr[0] = 0, rowptr[i+1] = rowptr[i] + counts[i]
 *   stream  cudaStream_t the work is enqueued on (NULL = legacy default stream); the call
 *           returns without waiting.
 * Limit: n <= 33,554,432 rows; a larger n fails with FEA_ERR_TOO_LARGE and does no work.
 * It calls no cudaMalloc, cudaFree or allocating library routine.  Its partial sums live in
 * one fixed 128 KiB array per GPU that every call in the process shares; each call rewrites
 * the part it uses, so nothing has to be cleared, but calls whose work overlaps on the GPU
 * (other streams, other threads) race on that array and must be serialised by the caller.
 * The first call on each GPU looks up the array's device address with that GPU current and
 * keeps it for the life of the process; make that first call before any stream capture, and
 * do not call this function again on a GPU after cudaDeviceReset in the same process (the
 * kept address would belong to the destroyed context).
 */
FEA_API fea_status fea_csr_rowptr_noalloc(const int32_t* counts, int64_t n, int64_t* rowptr, void* stream);

/*
 * fea_update_fields -- one step's change of the nodal field phi_old: a smooth seeded
 * perturbation, in place,
 *     phi[q][n] += A_q sin(kx_q x_n + ky_q y_n + kz_q z_n + psi_q)   (FP32),
 * x_n the node's coordinates.  The paper steps its transport fields in time (Sec. 2) and
 * reassembles every step; this perturbation stands in for the solver's update so that a
 * run of steps sees changing fields.
 *   phi     [n_eq][n_node] float DEVICE pointer, updated in place
 *   params  [n_eq][5] float DEVICE pointer: A, kx, ky, kz, psi per equation (the caller
 *           draws them; they are inputs, not generated here)
 * Enqueued on the mesh's stream.
 */
FEA_API fea_status fea_update_fields(fea_mesh* mesh, void* phi, int32_t n_eq, const float* params);

/*
 * fea_graph_capture_steps -- records n_steps time steps, each "fea_assemble, then
 * fea_update_fields with params + 5 n_eq s" (s = 0 .. n_steps-1), into one CUDA graph.
 * Arguments are those of fea_assemble (FP32 precision only; accumulate must be 0), plus
 *   params   [n_steps][n_eq][5] float DEVICE pointer, read at every launch
 * Every pointer is baked into the graph: the arrays must stay allocated, and their
 * contents at launch time are what the steps use.  Before recording, one eager assembly
 * runs (it builds the schedules and scratch, which cannot be captured) and waits; its
 * values/rhs are overwritten by the graph.  On success *out owns the graph.
 */
FEA_API fea_status fea_graph_capture_steps(fea_mesh* mesh, const fea_pattern* pattern, const void* velocity,
                                           const void* diffusivity, const void* reaction, void* phi_old, double dt,
                                           int32_t n_eq, const fea_assemble_opts* opts, void* values, void* rhs,
                                           const float* params, int32_t n_steps, fea_graph** out);
/* Launches the recorded steps on the mesh's current stream; returns without waiting. */
FEA_API fea_status fea_graph_launch(fea_graph* graph);
/* Frees the graph (the caller makes sure no launch of it is still running). */
FEA_API fea_status fea_graph_destroy(fea_graph* graph);

/*
 * fea_spmv -- y_q = A_q x_q for the n_eq FP32 matrices assembled on this pattern (the
 * operator the solver of Sec. 2 applies in its PCG).  The pattern's column indices are read
 * once per row for all equations.
 *   values [n_eq][nnz], x and y [n_eq][n_node] float DEVICE pointers; accumulate != 0 adds
 *   into y.  Enqueued on `stream` (cudaStream_t, NULL = legacy default stream).
 */
FEA_API fea_status fea_spmv(const fea_pattern* pattern, const float* values, const float* x, float* y, int32_t n_eq,
                            int32_t accumulate, void* stream);

/*
 * fea_pcg -- Jacobi-preconditioned conjugate gradients (Sec. 2, Alg. 1: the algebraic solver
 * is a preconditioned CG) on the n_eq FP32 matrices assembled on this pattern, each solved
 * for its own right-hand side: A_q x_q = b_q.  Every A_q must be symmetric positive
 * definite, e.g. an assembly with the MASS and DIFF terms only.
 *   values [n_eq][nnz], b [n_eq][n_node] float DEVICE pointers;
 *   x [n_eq][n_node] float DEVICE pointer: the initial guess in, the solution out.
 *   Equation q stops when ||b_q - A_q x_q||_2 <= rtol ||b_q||_2 or after max_iter iterations.
 *   iters [n_eq] (host, may be NULL): iterations taken; rel_resid [n_eq] (host, may be NULL):
 *   the final ||r_q||_2 / ||b_q||_2 of the recursively updated residual.
 * The equations iterate together, with FP32 vectors and FP64 scalars.  Runs on `stream` and
 * waits for it.  A diagonal entry or p.Ap <= 0 stops that equation and returns FEA_ERR_ARG
 * after the others finish.
 */
FEA_API fea_status fea_pcg(const fea_pattern* pattern, const float* values, const float* b, float* x, int32_t n_eq,
                           int32_t max_iter, double rtol, int32_t* iters, double* rel_resid, void* stream);

/*
 * fea_tuned_strategy -- the scatter (fea_scatter) and equation-group count that
 * FEA_SCATTER_AUTO settled on for this pattern and n_eq (full operator).  FEA_ERR_STATE if no
 * FP32 FEA_SCATTER_AUTO call has tuned that equation count yet.  Host only; does not wait.
 */
FEA_API fea_status fea_tuned_strategy(const fea_pattern* pattern, int32_t n_eq, int32_t* scatter, int32_t* eq_groups);

/*
 * fea_tuned_config -- every dimension FEA_SCATTER_AUTO settled on for this pattern, n_eq and
 * term mask (terms: FEA_TERM_* bits as passed in opts).  FEA_ERR_STATE before the first such
 * call.  Host only; does not wait.
 * The tuning cache: a JSON file, one object whose keys name the GPU, the element type (or
 * "mixed"), n_eq, the term mask and the mesh size class (element and node counts rounded to
 * powers of two), each mapped to a fea_tuning.  Its path is the environment variable
 * FEA_TUNE_CACHE, else $XDG_CACHE_HOME/fea_gb300/tuning.json, else
 * $HOME/.cache/fea_gb300/tuning.json; FEA_TUNE_CACHE=off disables it.  A tuned choice is
 * merged into the file (written to a temporary file, then renamed); a later process that
 * meets the same key uses the stored choice without timing.  A file that cannot be read or
 * written is ignored.
 */
FEA_API fea_status fea_tuned_config(const fea_pattern* pattern, int32_t n_eq, int32_t terms, fea_tuning* out);

/*
 * fea_tune_candidates -- the configurations FEA_SCATTER_AUTO may time for this pattern, n_eq
 * and term mask (every one is a valid explicit setting of opts): up to cap of them into out
 * (host array), their number in *count.  Host only; builds no schedule and launches nothing.
 */
FEA_API fea_status fea_tune_candidates(const fea_pattern* pattern, int32_t n_eq, int32_t terms, fea_tuning* out,
                                       int32_t cap, int32_t* count);

/*
 * fea_cancel_rows -- the cancellation check (opts.cancel_check = 1, FP32 path).  Row i of an
 * equation is flagged when an entry with |A_ij| > 1e-3 max_j |A_ij| has
 * sum_e |A^e_ij| > 1e3 |A_ij|, or when sum_e |b^e_i| > 1e3 |b_i| (the sums over the elements
 * containing the row's node); a row is flagged if any equation flags it.  Every checked
 * assembly computes the flags from its own inputs, in one FP32 pass over all rows, then
 * recomputes the flagged rows after the main assembly: element rows formed and summed in FP64
 * from the same inputs, rounded into the outputs.  The check is device work on the mesh's
 * stream, with no host wait, so checked assemblies can be recorded in a step graph; the first
 * checked assembly for a pattern and n_eq allocates the check's buffers and must come before
 * any stream capture.  The flag pass costs several times the element work of the assembly.
 * *count = the number of rows the most recent checked assembly for this n_eq flagged (the call
 * waits for the mesh's stream); FEA_ERR_STATE before the first checked call.
 */
FEA_API fea_status fea_cancel_rows(const fea_pattern* pattern, int32_t n_eq, int64_t* count);

/* Thread-local message describing the last failure of a call on this thread. */
FEA_API const char* fea_last_error(void);
/* Number of CUDA kernels this library has launched in this process so far. */
FEA_API int64_t fea_kernel_launches(void);
/* Library version, major*10000 + minor*100 + patch. */
FEA_API int32_t fea_version(void);

#ifdef __cplusplus
}
#endif
#endif /* FEA_H */
