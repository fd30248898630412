/*
 * ckks_kan.h — C ABI of the GB300 RNS-CKKS / encrypted-KAN library.
 *
 * Protocol (paper, Introduction and Threat Model): the client holds the
 * secret key, raster-scans and encrypts its input x (length n_i), the server
 * evaluates the KAN on the ciphertext with plaintext weights, and the client
 * decrypts the n_o outputs from slots [0, n_o).
 *
 * Conventions for every entry point:
 *  - Return value: CKKS_OK (0) or a negative CKKS_ERR_* code; no call aborts
 *    or throws across the ABI. ckks_strerror() names a code; ckks_last_error()
 *    gives the last failure's message on the calling thread.
 *  - Handles (ckks_ctx, ckks_keys, ckks_ct, kan_model) are opaque and
 *    library-owned; every `**out` handle is freed by its *_destroy call.
 *    Ciphertext and key data live in device (HBM) memory on the context's
 *    device.
 *  - Host arrays passed in are caller-owned and only read (or written, for
 *    outputs) during the call.
 *  - Device pointers (uint64_t* d_...) must point into memory on the
 *    context's device; the library does not take ownership.
 *  - Work is queued on the context's stream; calls that return host data
 *    (decrypt, export) synchronize that stream first.
 *  - A ciphertext handle holds a batch of B >= 1 ciphertexts at one level l
 *    (l + 1 RNS limbs), laid out [B][2][l+1][N] uint64 in NTT form.
 */
#ifndef CKKS_KAN_H
#define CKKS_KAN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CKKS_OK 0
#define CKKS_ERR_INVALID_ARG -1
#define CKKS_ERR_LEVEL -2        /* level exhausted or levels not compatible */
#define CKKS_ERR_SCALE -3        /* operand scales differ by more than 2^-30 */
#define CKKS_ERR_MISSING_KEY -4  /* no Galois key for a requested rotation */
#define CKKS_ERR_OUT_OF_MEMORY -5
#define CKKS_ERR_CUDA -6
#define CKKS_ERR_OVERFLOW -7     /* a value does not fit its encoding scale */
#define CKKS_ERR_TIMEOUT -8       /* a time-bounded wait ran out (device or serving) */
#define CKKS_ERR_UNSUPPORTED -9

typedef struct ckks_ctx ckks_ctx;
typedef struct ckks_keys ckks_keys;
typedef struct ckks_ct ckks_ct;
typedef struct kan_model kan_model;
typedef struct ckks_lt ckks_lt;
typedef struct ckks_boot ckks_boot;

const char* ckks_strerror(int code);
const char* ckks_last_error(void);

/* ------------------------------------------------------------ context
 * RNS-CKKS parameters (the scheme the paper builds on, HE section; the
 * parameter rules are this library's own):
 *   N = 2^log_n; q_0 = largest prime < 2^q0_bits with q_0 = 1 mod 2N;
 *   n_special special primes below 2^p_bits; n_scale rescaling primes,
 *   chosen top-down so that the canonical scale of level l,
 *   Delta_L = 2^scale_bits, Delta_{l-1} = Delta_l^2 / q_l, stays at ~2^scale_bits.
 * Key switching is hybrid with digits of n_special consecutive Q primes.
 * device: CUDA ordinal. Errors: INVALID_ARG on out-of-range sizes
 * (2 <= log_n <= 16, n_special >= 1, bit sizes <= 61), CUDA on device errors. */
int ckks_context_create(int log_n, int q0_bits, int scale_bits, int n_scale, int p_bits,
                        int n_special, int device, ckks_ctx** out);
int ckks_context_destroy(ckks_ctx* ctx);
/* Hybrid key-switching digit layout by measurement (no counterpart in the
 * paper, which delegates key switching to SEAL). For the chain q0_bits +
 * n_scale x scale_bits and a bound max_qp_bits on log2(QP) (the security
 * budget), every alpha in {1, 2, 3, 4, 5, 6, 8, 10, 12} takes special primes
 * of p_bits = min(60, floor((max_qp_bits - log2 Q) / alpha)) bits and is kept
 * if p_bits >= 30 and alpha p_bits >= q0_bits + (alpha - 1) scale_bits (P
 * covers the largest digit). Each kept layout builds a context on `device`,
 * and times 3 x (HMult + HRot) of `batch` ciphertexts at the top level.
 * Out: the fastest alpha and its p_bits; tried[i], ms[i] (ms per HMult+HRot)
 * for the first `cap` layouts timed; *n_tried their count (all may be NULL
 * but alpha and p_bits). UNSUPPORTED if no layout fits. */
int ckks_autotune_keyswitch(int log_n, int q0_bits, int scale_bits, int n_scale, int max_qp_bits,
                            int batch, int device, int* alpha, int* p_bits, int* tried,
                            double* ms, int cap, int* n_tried);
/* moduli: n_qp = n_scale + 1 + n_special words (q_0..q_L, p_0..); delta: n_scale + 1
 * canonical scales; either may be NULL. */
int ckks_context_info(const ckks_ctx* ctx, uint64_t* moduli, double* delta, int* n_qp);
/* Queue work on `stream` (a cudaStream_t) instead of the library's own stream. */
int ckks_set_stream(ckks_ctx* ctx, void* stream);
/* Kernel fusion on (default, enabled != 0) or off. On: ModUp's basis
 * conversion, ModDown's and rescale's subtract-and-scale run inside the
 * NTT kernels' loads and stores (N = 2^13 .. 2^16). Off: separate
 * conversion, transform and pointwise launches, the plain form. Results are
 * identical word for word either way; only speed changes. */
int ckks_set_fusion(ckks_ctx* ctx, int enabled);
/* Waits for the context's stream. Kernels that wait on asynchronous copies
 * (the TMA-staged key inner product of every key switch) bound each wait to
 * about two seconds; one that runs out records it in a device status word,
 * leaves its outputs unwritten and returns. ckks_synchronize then returns
 * CKKS_ERR_TIMEOUT (once; the word is cleared): every result computed since
 * the previous ckks_synchronize is invalid, the context stays usable. */
int ckks_synchronize(ckks_ctx* ctx);
/* Self-test of that path: one CTA waits, with a limit of limit_cycles SM
 * clock cycles (1 .. 2^32), on an mbarrier phase that nothing completes.
 * Returns CKKS_ERR_TIMEOUT when the wait ran out and was reported as above
 * (the expected result), CKKS_OK if it was not. */
int ckks_selftest_wait(ckks_ctx* ctx, long long limit_cycles);

/* ------------------------------------------------------------ raw kernels
 * Forward (inverse != 0: inverse) negacyclic NTT of n_rows rows of N uint64
 * at device pointer d_rows, row r reduced mod q_{r % limbs}. Forward output
 * is bit-reversed: A[j] = sum_i a[i] psi^((2 brv(j)+1) i) mod q, where psi is
 * the first x^((q-1)/2N), x = 2,3,..., with psi^N = -1. Inputs must be < q. */
int ckks_ntt(ckks_ctx* ctx, uint64_t* d_rows, size_t n_rows, int limbs, int inverse);

/* ------------------------------------------------------------ launch accounting
 * Every kernel launch is counted per kind (names from ckks_kernel_kind_name,
 * kinds 0 .. ckks_kernel_kind_count()-1; the last kind counts device copies,
 * not kernels). With profiling on, each launch is also bracketed by CUDA
 * events on the context's stream; ckks_profile_collect synchronizes, then
 * writes per kind the summed event time (ms), the summed algorithmic bytes
 * (the minimum HBM traffic of the launch: inputs read once, outputs written
 * once) and the number of timed launches, and clears the records. */
int ckks_kernel_kind_count(void);
const char* ckks_kernel_kind_name(int kind);
int ckks_launch_counts(const ckks_ctx* ctx, uint64_t* counts, int cap);
int ckks_profile_enable(ckks_ctx* ctx, int on);
int ckks_profile_collect(ckks_ctx* ctx, double* ms, double* bytes, uint64_t* launches, int cap);
/* Same, plus per kind the summed algorithmic count of 64-bit modular
 * multiplications (NTT butterflies, basis-conversion and scaling products,
 * key inner-product products); modmuls may be NULL. */
int ckks_profile_collect2(ckks_ctx* ctx, double* ms, double* bytes, double* modmuls,
                          uint64_t* launches, int cap);
/* Measured integer-pipe peak of the context's device (the denominator of the
 * integer roofline; the paper has no counterpart): register-only chains of
 * kind 0, 64 x 64 -> 128-bit products (low and high words), *per_s in
 * products/s; kind 1, the forward NTT's lazy butterfly (three-product Shoup
 * multiply and both sums, one full reduction of each word per 16 stages),
 * in butterflies/s; kind 2, the three-product Shoup multiply alone (the
 * basis-conversion product), in products/s. Timed with CUDA events over
 * several launches of SMs x resident-blocks CTAs on the context's stream. */
int ckks_int_peak(ckks_ctx* ctx, int kind, double* per_s);

/* NTT launch shape (the paper has no counterpart; an implementation
 * choice of the transforms): the clustered 2^15- and 2^16-point transforms
 * run at 2 CTAs per SM (64 registers per thread) or 1 (up to 128), per slot:
 * 0 plain forward, 1 ModUp, 2 ModDown, 3 rescale, 4 HMult's merged
 * relinearise-rescale division, 5 inverse. ckks_autotune_ntt times a batch
 * of `batch` ciphertexts at the top level (HMult, HRot, a constant product,
 * a rescale, a plain forward transform) under both settings with per-launch
 * CUDA events and keeps the faster per slot on the context (results are the
 * same words either way); ms[0..5] are the slots' times at 2 CTAs per SM,
 * ms[6..11] at 1, chosen[0..5] the kept setting (either may be NULL). Other
 * ring sizes keep 2. ckks_set_ntt_shape sets one slot. */
int ckks_autotune_ntt(ckks_ctx* ctx, int batch, double* ms, int* chosen);
int ckks_set_ntt_shape(ckks_ctx* ctx, int slot, int ctas_per_sm);

/* ------------------------------------------------------------ keys
 * Secret-key generation from `seed` (ternary secret, ChaCha20 stream), the
 * relinearisation key, and one Galois key per rotation step in rot_steps
 * (Eq. 10: step t > 0 rotates left). Key data: [digit][2][n_qp][N]. */
int ckks_keygen(ckks_ctx* ctx, uint64_t seed, const int32_t* rot_steps, size_t n_steps,
                ckks_keys** out);
int ckks_keys_destroy(ckks_keys* keys);
/* Copy the secret key (NTT form, n_qp x N words) or a switching key
 * (galois = 0: relinearisation; beta_max x 2 x n_qp x N words) to host. */
int ckks_keys_export_secret(const ckks_keys* keys, uint64_t* host, size_t cap_words);
int ckks_keys_export_switch(const ckks_keys* keys, uint64_t galois, uint64_t* host,
                            size_t cap_words);
/* Galois element of a left rotation by `step`: 5^(step mod N/2) mod 2N. */
uint64_t ckks_galois_element(const ckks_ctx* ctx, int32_t step);

/* ------------------------------------------------------------ ciphertexts
 * Encrypt `batch` vectors of n <= N/2 real values (values[b*n + j]) at
 * `level` with scale Delta_level: c0 = -a s + m + e, c1 = a, where m is the
 * canonical-embedding encoding, a ~ U(Z_q) and e centred-binomial (eta = 21),
 * drawn from ChaCha20 streams keyed by `seed` and object id first_index + b.
 * Errors: OVERFLOW if a value does not fit the scale. */
int ckks_encrypt(ckks_ctx* ctx, const ckks_keys* keys, const double* values, size_t batch,
                 size_t n, int level, uint64_t seed, uint64_t first_index, ckks_ct** out);
/* Decrypt to host: out[b*n + j], n <= N/2. Uses limb 0 only, which is exact
 * while |scale * value| < q_0 / 2. */
int ckks_decrypt(ckks_ctx* ctx, const ckks_keys* keys, const ckks_ct* ct, double* out,
                 size_t n);
int ckks_ct_info(const ckks_ct* ct, size_t* batch, int* level, double* scale);
/* Host copy of the batch, [B][2][level+1][N] words; cap_words must be >= that. */
int ckks_ct_export(const ckks_ct* ct, uint64_t* host, size_t cap_words);
int ckks_ct_import(ckks_ctx* ctx, const uint64_t* host, size_t batch, int level, double scale,
                   ckks_ct** out);
/* Asynchronous import for pipelining inputs with computation: the copy (and
 * the device allocation) run in the order of `copy_stream` (a cudaStream_t),
 * and the library's stream waits for the copy before any later work, so the
 * copy of the next batch overlaps the computation of the current one. The
 * caller keeps `host` (pinned memory for true asynchrony) unchanged until the
 * copy has completed (e.g. until copy_stream is synchronized). */
int ckks_ct_import_async(ckks_ctx* ctx, const uint64_t* host, size_t batch, int level,
                         double scale, void* copy_stream, ckks_ct** out);
/* Sub-batch [first, first+count) of a batch, copied. */
int ckks_ct_slice(ckks_ctx* ctx, const ckks_ct* ct, size_t first, size_t count, ckks_ct** out);
int ckks_ct_destroy(ckks_ct* ct);

/* ------------------------------------------------------------ homomorphic ops
 * Eq. 6 / 7: slot-wise add / subtract. Equal batch, level and scale. */
int ckks_add(ckks_ctx* ctx, const ckks_ct* a, const ckks_ct* b, ckks_ct** out);
int ckks_sub(ckks_ctx* ctx, const ckks_ct* a, const ckks_ct* b, ckks_ct** out);
/* Eq. 8 without rescale: tensor product then relinearisation (hybrid key
 * switch of the s^2 component). Equal batch and level; scale = product. */
int ckks_mul_relin(ckks_ctx* ctx, const ckks_keys* keys, const ckks_ct* a, const ckks_ct* b,
                   ckks_ct** out);
/* Divide by the top prime q_l with centred rounding; level - 1. */
int ckks_rescale(ckks_ctx* ctx, const ckks_ct* in, ckks_ct** out);
/* The same rescale for callers that cannot allocate device memory (for
 * example while a stream is being captured, or under a fixed memory budget);
 * the paper has no counterpart. Computes exactly what ckks_rescale computes,
 * on raw device buffers: d_in holds `batch` ciphertexts [batch][2][level+1][N]
 * in NTT form at `level` (>= 1), d_out receives [batch][2][level][N]; the
 * output scale is the input scale / q_level (the caller keeps the scale).
 * Both buffers are caller-owned device memory on the context's device; work
 * is queued on the context's stream. No allocation happens: the working
 * memory is a fixed 64 MiB device array inside the library (8 Mi words, held
 * by every GPU that loads the library until exit); sizes needing more than
 * 2 * batch * N * (level + 1) <= 8 Mi words are rejected with
 * CKKS_ERR_INVALID_ARG. d_in and d_out must not overlap (the output's limb
 * stride differs from the input's); overlapping buffers are rejected with
 * CKKS_ERR_INVALID_ARG. The first call on a device looks the array up (do it
 * before any stream capture). All calls share the array: calls that overlap
 * on the GPU race, so serialize them. The calling thread's current device is
 * left as it was. */
int ckks_rescale_noalloc(ckks_ctx* ctx, const uint64_t* d_in, size_t batch, int level,
                         uint64_t* d_out);
/* Eq. 8 complete: bring both to the lower level, multiply, relinearise and
 * rescale. The relinearisation's division by P and the rescale's division by
 * q_level are one rounded division by P q_level (centred basis conversion of
 * the dropped limbs), level - 1 on output. */
int ckks_mul(ckks_ctx* ctx, const ckks_keys* keys, const ckks_ct* a, const ckks_ct* b,
             ckks_ct** out);
/* Eq. 9: slot-wise product with real vector v (n values, rest 0) encoded at
 * the scale that lands on Delta_{l-1} after the included rescale. */
int ckks_mul_plain(ckks_ctx* ctx, const ckks_ct* a, const double* v, size_t n, ckks_ct** out);
/* a + v slot-wise (v encoded at a's scale). */
int ckks_add_plain(ckks_ctx* ctx, const ckks_ct* a, const double* v, size_t n, ckks_ct** out);
/* a * c (real scalar, rescaled) and a + c. */
int ckks_mul_const(ckks_ctx* ctx, const ckks_ct* a, double c, ckks_ct** out);
int ckks_add_const(ckks_ctx* ctx, const ckks_ct* a, double c, ckks_ct** out);
/* Move to a lower level with the canonical scale Delta_level. */
int ckks_level_down(ckks_ctx* ctx, const ckks_ct* a, int level, ckks_ct** out);
/* Eq. 10: rotate left by `step` slots (right for step < 0). */
int ckks_rotate(ckks_ctx* ctx, const ckks_keys* keys, const ckks_ct* in, int32_t step,
                ckks_ct** out);
/* Several rotations of one input sharing a single ModUp (hoisting);
 * outs[i] receives the rotation by steps[i]; bit-identical to ckks_rotate. */
int ckks_rotate_hoisted(ckks_ctx* ctx, const ckks_keys* keys, const ckks_ct* in,
                        const int32_t* steps, size_t n_steps, ckks_ct** outs);

/* ------------------------------------------------------------ bootstrapping
 * The paper's parameter sets bootstrap as in Lee et al. 2022 (Experiment
 * Setup): ModRaise, CoeffToSlot, EvalMod, SlotToCoeff. Slot j of the
 * encoder holds sum_i w_i zeta_j^i, w_i = m_i + i m_(i+N/2),
 * zeta_j = exp(i pi 5^j / N); rot(x, t) moves slot j + t to slot j.
 *
 * Keys with a sparse ternary secret of Hamming weight `hamming_weight`
 * (0: the dense ternary secret of ckks_keygen, identical keys) and, if
 * `conjugation`, the key of the Galois element 2N - 1 (X -> X^-1, the
 * slots' complex conjugates). Sparse draw: partial Fisher-Yates shuffle on
 * the ChaCha20 stream (seed, domain 4, id 0), step i swapping position i
 * with i + w32[2i] mod (N - i) and giving the drawn position the sign -1 if
 * w32[2i+1] is odd, else +1. public_seed != 0 (and != seed) draws the
 * switching keys' uniform halves from that public seed instead of `seed`
 * (needed by ckks_keys_compress); 0 keeps ckks_keygen's keys. */
int ckks_keygen_ex(ckks_ctx* ctx, uint64_t seed, int hamming_weight, const int32_t* rot_steps,
                   size_t n_steps, int conjugation, uint64_t public_seed, ckks_keys** out);
/* Seed-compressed switching keys (the BSGS section's keys; NEXT-4): a key
 * pair (b, a) keeps only b, and a is regenerated on the device before each
 * key switch from the public seed (ChaCha20 stream (public_seed, domain 3,
 * object 2^40 | g << 8 | j), as at key generation), so every result is
 * word for word the uncompressed keys'. The resident switching-key bytes
 * halve; each key switch pays the regeneration (beta_max n_qp limbs of
 * ChaCha20 output and two copies) in scratch device memory. Only keys made
 * by ckks_keygen_ex with a public_seed (nonzero, different from the seed)
 * can be compressed: otherwise the uniform halves come from the secret's
 * seed, and handing that out would reveal the secret (CKKS_ERR_INVALID_ARG).
 * Irreversible; ckks_keys_export_switch then exports the regenerated key. */
int ckks_keys_compress(ckks_keys* keys);
/* Device bytes the key set holds (secret and switching keys). */
int ckks_keys_bytes(const ckks_keys* keys, size_t* bytes);
/* ModRaise: a level-0 batch read over limbs 0..level (the centred residues
 * mod q0 of each coefficient reduced mod every q_t); same scale.
 * CKKS_ERR_LEVEL unless `in` is at level 0 and level <= L. */
int ckks_mod_raise(ckks_ctx* ctx, const ckks_ct* in, int level, ckks_ct** out);
/* X -> X^(2N-1) (the conjugation key is needed): slots conjugated. */
int ckks_conjugate(ckks_ctx* ctx, const ckks_keys* keys, const ckks_ct* in, ckks_ct** out);
/* Times the monomial X^k (k taken mod 2N): exact, no level. Slot j is
 * multiplied by zeta_j^k; X^(N/2) multiplies every slot by i. */
int ckks_mul_monomial(ckks_ctx* ctx, const ckks_ct* in, int64_t k, ckks_ct** out);
/* Times a constant far below 1 (two levels, canonical scale of level - 2):
 * the integer rint(value S2), S2 = Delta_(l-2) q_l q_(l-1) / scale, of any
 * size, applied by its residues, then two rescales. CKKS_ERR_LEVEL below
 * level 2. */
int ckks_mul_const_wide(ckks_ctx* ctx, const ckks_ct* in, double value, ckks_ct** out);

/* A slot linear transform z -> sum_k d_k (.) rot(z, base + k stride),
 * k < n_diag, for inputs at `level` with scale `in_scale` (0: Delta_level);
 * re / im: host [n_diag][N/2] real and imaginary parts of the diagonals (an
 * all-zero diagonal is skipped), copied and encoded at creation (device
 * plaintexts [nonzero][level+1][N], over QP_level for form 1). Applied by
 * baby-step giant-step with g1 baby steps (0: the least power of two whose
 * square is >= n_diag for form 0, >= 4 n_diag for form 1, whose baby steps
 * cost no ModDown): it takes one level and lands on the canonical
 * scale. form 0: hoisted baby rotations, one rescale per giant step; form 1:
 * double hoisting, the baby rotations kept in QP_level and each giant step's
 * products divided by P q_level once (the rounding differs from form 0).
 * Rotation keys: see ckks_lt_rotations. */
int ckks_lt_create(ckks_ctx* ctx, int level, double in_scale, int64_t base, int64_t stride,
                   size_t n_diag, const double* re, const double* im, int g1, int form,
                   ckks_lt** out);
int ckks_lt_destroy(ckks_lt* lt);
/* Rotation steps the transform uses (baby steps j stride, giant steps
 * base + g1 i stride, mod N/2, without 0); *n receives their count. */
int ckks_lt_rotations(const ckks_lt* lt, int32_t* steps, size_t cap, size_t* n);
/* CKKS_ERR_LEVEL / CKKS_ERR_SCALE if `in` is not at the transform's level
 * and input scale; CKKS_ERR_MISSING_KEY for a missing rotation key. */
int ckks_lt_apply(ckks_ctx* ctx, const ckks_keys* keys, const ckks_lt* lt, const ckks_ct* in,
                  ckks_ct** out);

/* A bootstrapping plan computed by the library: overflow bound K (the
 * ModRaise multiple |I| <= K), EvalMod by the Chebyshev interpolant of
 * degree `degree` of (c / 2 pi) sin(2 pi 2^e y / c), c = q0 / Delta_0,
 * 2^e >= (K + 1) c; CoeffToSlot and SlotToCoeff as cts_levels and
 * stc_levels merged levels of the special-FFT stages (log2(N/2) stages in
 * near-equal groups), in the transform form `form` (ckks_lt_create).
 * CoeffToSlot starts at level L on inputs of scale
 * Delta_0; the output comes out at L - cts_levels - 2 - depth(degree) -
 * stc_levels. CKKS_ERR_LEVEL if the chain is too short. */
int ckks_boot_create(ckks_ctx* ctx, int K, int degree, int cts_levels, int stc_levels, int form,
                     ckks_boot** out);
/* The same from given parts: exponent e, EvalMod's Chebyshev coefficients,
 * the CoeffToSlot and SlotToCoeff transforms in application order (borrowed:
 * they must outlive the plan). */
int ckks_boot_create_ex(ckks_ctx* ctx, int e, const double* cheb, size_t n_cheb,
                        const ckks_lt* const* cts, size_t n_cts, const ckks_lt* const* stc,
                        size_t n_stc, ckks_boot** out);
int ckks_boot_destroy(ckks_boot* boot);
/* e, the level CoeffToSlot and SlotToCoeff start at, the number of
 * Chebyshev coefficients (each pointer may be NULL). */
int ckks_boot_info(const ckks_boot* boot, int* e, int* cts_level, int* stc_level,
                   size_t* n_cheb);
int ckks_boot_coefficients(const ckks_boot* boot, double* cheb, size_t cap);
/* base, stride and diagonal count of transform `index` (inverse != 0:
 * CoeffToSlot). */
int ckks_boot_diagonals(const ckks_boot* boot, int inverse, size_t index, int64_t* base,
                        int64_t* stride, size_t* n_diag);
/* The library's merged levels for n_levels groups (inverse != 0: the
 * CoeffToSlot factors 2 F^-1): level `index`'s base, stride, count and, if
 * re and im are given, its diagonals ([n_diag][N/2], cap doubles each). */
int ckks_boot_levels(ckks_ctx* ctx, int n_levels, int inverse, size_t index, double* re,
                     double* im, size_t cap, int64_t* base, int64_t* stride, size_t* n_diag);
/* Every rotation step of the plan's transforms (keys for ckks_keygen_ex,
 * with conjugation). */
int ckks_boot_rotations(const ckks_boot* boot, int32_t* steps, size_t cap, size_t* n);
/* The steps one by one: CoeffToSlot of a raised batch into the two real-slot
 * halves y_lo, y_hi (slot p holding t_(brv(p)) / (Delta_0 2^e) and
 * t_(N/2 + brv(p)) / (Delta_0 2^e)); EvalMod of one half; SlotToCoeff of the
 * two reduced halves. */
int ckks_boot_coeff_to_slot(ckks_ctx* ctx, const ckks_keys* keys, const ckks_boot* boot,
                            const ckks_ct* raised, ckks_ct** lo, ckks_ct** hi);
int ckks_boot_eval_mod(ckks_ctx* ctx, const ckks_keys* keys, const ckks_boot* boot,
                       const ckks_ct* in, ckks_ct** out);
int ckks_boot_slot_to_coeff(ckks_ctx* ctx, const ckks_keys* keys, const ckks_boot* boot,
                            const ckks_ct* lo, const ckks_ct* hi, ckks_ct** out);
/* The whole refresh of a level-0 batch: ModRaise to the CoeffToSlot level,
 * CoeffToSlot, EvalMod of both halves, SlotToCoeff; the slots come back up
 * to the plan's precision at the level ckks_boot_create states. */
int ckks_bootstrap(ckks_ctx* ctx, const ckks_keys* keys, const ckks_boot* boot,
                   const ckks_ct* in, ckks_ct** out);

/* ------------------------------------------------------------ encrypted KAN
 * One KAN layer (paper, Method): n_in -> n_out with a uniform grid of G
 * intervals on [grid_lo, grid_hi] and order-k B-splines (Eqs. 1-4), spline
 * coefficients coef[o][i][m] (m < G+k), spline scaler w_s[o][i] and base
 * weights w_b[o][i]; the HE-friendly parameters are the comparison bound R
 * (Algorithm 2), the SiLU polynomial (Eqs. 11-12) as Chebyshev coefficients
 * on [silu_lo, silu_hi], and the comparison composite f_{comp[0]} o ... as
 * the orders n of f_n(x) = sum_i 4^-i C(2i,i) x (1-x^2)^i, or given by its
 * stages' coefficients (comp_poly). All arrays are row-major doubles, copied
 * at model creation. */
typedef struct {
  int n_in, n_out, G, k;
  double grid_lo, grid_hi;
  const double* coef;
  const double* w_s;
  const double* w_b;
  double R;
  double silu_lo, silu_hi;
  const double* silu_cheb;
  int silu_degree;
  const int* comp;
  int n_comp;
  /* 0: lazy combination, the fused W_f = W'P of Eq. 13 on the ColTile basis.
   * 1: the naive method the paper compares against (Table 3): an HE matvec by
   * the permutation P of Algorithm 3 (n_i(g+k) diagonals, one more level),
   * then W' on the row-major basis. */
  int naive;
  /* Explicit comparison composite, used instead of comp when n_comp_poly > 0
   * (comp may then be NULL): stage s, applied in order, is the odd polynomial
   * sum_l c_l u^(2l+1) with the comp_poly_len[s] coefficients c_0, c_1, ..
   * read in turn from comp_poly (for example from kan_comp_minimax); the
   * last stage returns (1 + p) / 2. Stages of at most 32 coefficients. */
  const double* comp_poly;
  const int* comp_poly_len;
  int n_comp_poly;
  /* Order-0 basis of Algorithm 2. 0: the product B_{m,0} =
   * PolyComp(x - t_m) PolyComp(t_{m+1} - x), as the algorithm prints it.
   * 1: the difference B_{m,0} = s_m - s_{m+1}, s_m = PolyComp(x - t_m) over
   * all g + 2k + 1 knots and s_{m+1} = rot(s, n_i): one comparison and no
   * product (one level fewer); equal to the product form for exact
   * comparisons since PolyComp(-a) = 1 - PolyComp(a) for an odd composite.
   * Algorithm 1 then packs 2^ceil(log2(g + 2k + 1)) copies. */
  int b0_form;
  /* Matvec form (the Lazy combination section's BSGS): 0 = baby-step
   * rotations hoisted (one ModUp, a ModDown each); 1 = double hoisting: the
   * baby steps stay in QP_l, the diagonal products of a giant step are summed
   * over QP_l and divided by P q_l once (ModDown and rescale in one rounded
   * division). Not for a chunked first layer (UNSUPPORTED). */
  int bsgs_form;
} kan_layer_desc;

/* PolyComp by composite minimax polynomials (Algorithm 2 cites Lee et al.'s
 * minimax composites without degrees): stage 1 is the odd polynomial of
 * degree degrees[0] with the least maximum error against 1 on [eps, A]
 * (against sign on [-A, -eps] u [eps, A]; PolyComp's range is A = 1, and the
 * comparison bound R keeps calibration inputs within 1/1.1 of it); stage
 * s + 1 the same on the image
 * of stage s's interval; each by the Remez exchange over 40001 points. coef
 * receives the stages' odd monomial coefficients, (degrees[s] + 1) / 2 each,
 * in order (the layout of kan_layer_desc.comp_poly); taus (may be NULL) the
 * composite's maximum distance from 1 on [eps, A] after each stage. Odd
 * degrees 1..63; INVALID_ARG if a stage leaves values <= 0 (eps too small). */
int kan_comp_minimax(double eps, double A, const int* degrees, int n_stages, double* coef,
                     double* taus);

/* Host-only model preparation (no device work).
 * kan_silu_fit: Chebyshev coefficients cheb[0..degree] (basis of [lo, hi]
 * mapped to [-1, 1]) of the SiLU fit on n_samples evenly spaced points of
 * [lo, hi]: method KAN_FIT_WLS is Eq. 12 (weight 10 within mu +- 3 sigma, 1
 * outside), KAN_FIT_OLS unit weights (both by Householder QR), KAN_FIT_REMEZ
 * the minimax polynomial over the points by the Remez exchange.
 * kan_calibrate: for each layer (only n_in, n_out, G, k, grid, coef, w_s,
 * w_b, the comparison composite and b0_form of `layers` are read), the
 * statistics of the layer's inputs over the n calibration vectors
 * X[n][n_in] as the encrypted network computes
 * them (the HE-friendly FP64 KAN: fitted SiLU, PolyComp indicators with the
 * layer's comparison composite, the earlier layers already calibrated), the
 * SiLU range of Eq. 11 (or fixed_range[0..1] if not NULL) and its fit, and
 * the comparison bound R = 1.1 (max|x| + max|knot|) / 2 of Algorithm 2.
 * Outputs per layer: R[l], silu_lo[l], silu_hi[l], cheb[l*(degree+1) ..]. */
enum {
  KAN_FIT_WLS = 0,   /* Eq. 12: weight 10 within mu +- 3 sigma, 1 outside */
  KAN_FIT_OLS = 1,   /* least squares, unit weights (Table 5 comparison) */
  KAN_FIT_REMEZ = 2  /* minimax on [lo, hi] by the Remez exchange (Table 5) */
};
int kan_silu_fit(double lo, double hi, double mu, double sigma, int degree, int n_samples,
                 int method, double* cheb);
int kan_calibrate(const kan_layer_desc* layers, size_t n_layers, const double* X, size_t n,
                  int silu_degree, const double* fixed_range, int n_fit_samples, int fit_method,
                  double* R, double* silu_lo, double* silu_hi, double* cheb);

int kan_model_create(ckks_ctx* ctx, const kan_layer_desc* layers, size_t n_layers,
                     kan_model** out);
int kan_model_destroy(kan_model* model);
/* Rotation steps the schedule uses (pass them to ckks_keygen); *n receives
 * the count; at most cap are written. */
int kan_model_rotations(const kan_model* model, int32_t* steps, size_t cap, size_t* n);
/* Multiplicative depth (levels consumed) of one layer. */
int kan_model_layer_depth(const kan_model* model, int layer, int* depth);
/* Input chunking of one layer: when n_in * 2^J (J = ceil(log2(G + 2k)), or
 * ceil(log2(G + 2k + 1)) in the difference form, the repeat-packing factor
 * of Algorithm 1) exceeds the slots, the layer
 * takes *K > 1 input ciphertexts per request, each of *n_c consecutive inputs
 * (the last zero-padded), as consecutive batch elements; otherwise *K = 1 and
 * *n_c = n_in. Only layer 0 may be chunked. */
int kan_model_layer_chunks(const kan_model* model, int layer, int* K, int* n_c);
/* CUDA-graph replay of layer schedules on (enabled != 0) or off (default;
 * turning it off frees the captured graphs). With graphs on, kan_layer_eval,
 * kan_infer and the server run each layer, per input shape (batch, level,
 * scale) and key set, eagerly on the first call, capture the schedule into a
 * graph on the second and replay it afterwards; every temporary is
 * allocated inside the graph, the input and result pass through two
 * graph-owned buffers. Results are identical word for word to the eager
 * schedule. */
int kan_model_set_graphs(kan_model* model, int enabled);
/* Deeper networks than the chain holds: with a bootstrapping plan set
 * (borrowed; NULL clears it), kan_infer refreshes the batch before any layer
 * after the first whose depth (kan_model_layer_depth) exceeds the batch's
 * level. A batch of several ciphertexts with a level to spare is refreshed
 * packed: each ciphertext masked to the previous layer's n_out leading slots
 * (one level), packed by a rotation tree into one ciphertext per N/2 / nb
 * (nb the least power of two >= n_out; ciphertext b at slots b nb..),
 * brought to level 0 and bootstrapped, and unpacked by a rotation tree (the
 * next layer masks its input, so the other blocks do no harm); otherwise
 * each ciphertext is brought to level 0 and bootstrapped. The keys passed to
 * kan_infer then need the plan's rotations, the conjugation key and, for
 * packing, kan_model_refresh_rotations. */
int kan_model_set_bootstrap(kan_model* model, const ckks_boot* boot);
/* The rotation steps packed refreshes of a batch of `batch` take (+-s nb,
 * s = 1, 2, 4, .. below the ciphertexts per packed one, mod N/2). */
int kan_model_refresh_rotations(const kan_model* model, size_t batch, int32_t* steps, size_t cap,
                                size_t* n);
/* One layer on a batch: repeat packing (Algorithm 1), B-spline basis
 * (Algorithm 2), fused linear layer W_f = W'P (Algorithm 3, Eq. 13) and the
 * polynomial SiLU branch, both linear maps by BSGS diagonal matvec with
 * hoisted rotations. Output slots [0, n_out). */
int kan_layer_eval(ckks_ctx* ctx, const ckks_keys* keys, kan_model* model, int layer,
                   const ckks_ct* in, ckks_ct** out);
/* Whole network on n_in input handles (batches, any levels): inputs are moved
 * to the lowest level, concatenated into one batch and evaluated together.
 * A first layer whose repeat-packed input n_i 2^ceil(log2(G+2k)) exceeds N/2
 * takes K = ceil(n_i / n_c) ciphertexts per request, n_c = (N/2) /
 * 2^ceil(log2(G+2k)): ciphertext c holds inputs [c n_c, (c+1) n_c) (zero
 * beyond n_i), and the concatenated batch is request-major (element
 * r K + c); the K partial outputs of a request are summed, so the output
 * batch has one ciphertext per request. */
int kan_infer(ckks_ctx* ctx, const ckks_keys* keys, kan_model* model,
              const ckks_ct* const* in, size_t n_in, ckks_ct** out);

/* ------------------------------------------------------------ serving
 * Continuous batching of encrypted inference requests (the serving pattern
 * of the build; the paper itself times single inputs). Requests are admitted
 * first-come first-served while the sum of their device-memory footprints
 * stays within hbm_budget_bytes. A model's footprint per request is measured
 * by kan_server_add_model: the network runs once (after a run that fills the
 * model's plaintext caches) on a zero ciphertext at the top level, and the
 * rise of the device memory pool's used-bytes watermark is recorded (the
 * bytes a request needs beyond its input ciphertext; models are measured
 * and served with CUDA-graph replay off, the default). Each
 * kan_server_step evaluates one layer for every active request, batching
 * requests of the same model, layer and level into one evaluation; requests
 * submitted meanwhile join at the next step. Results are word-for-word those
 * of evaluating each request alone, or, for a model with a bootstrapping
 * plan (kan_model_set_bootstrap), those of kan_infer on the batch the
 * requests shared: a group whose level is below the next layer's depth is
 * refreshed as kan_infer refreshes a batch (packed when it holds several
 * requests), and the keys then need kan_model_refresh_rotations for the
 * largest group. kan_server_take returns CKKS_PENDING
 * while a request is still queued or running. The server does not own the
 * models or keys, which must outlive it. */
#define CKKS_PENDING 1
typedef struct kan_server kan_server;
int kan_server_create(ckks_ctx* ctx, size_t hbm_budget_bytes, kan_server** out);
int kan_server_destroy(kan_server* server);
/* Runs the model twice on the device to measure its footprint (above);
 * LEVEL if the model is deeper than the chain and has no bootstrapping plan
 * (with one, the first layer must fit). */
int kan_server_add_model(kan_server* server, kan_model* model, const ckks_keys* keys,
                         int* model_id);
/* The measured footprint of one request of the model, in bytes. */
int kan_server_footprint(const kan_server* server, int model_id, size_t* bytes);
/* `in` holds one request (batch 1 ciphertext, copied); errors: LEVEL if its
 * level is below the model's depth, OUT_OF_MEMORY if its footprint exceeds
 * the whole budget (it is refused, never admitted alone). */
int kan_server_submit(kan_server* server, int model_id, const ckks_ct* in, uint64_t* request_id);
int kan_server_step(kan_server* server, size_t* completed);
int kan_server_take(kan_server* server, uint64_t request_id, ckks_ct** out);
/* hbm_in_use / hbm_peak: the admitted footprints now / at most (never above
 * the budget); hbm_measured_peak: the largest rise of the device pool's used
 * bytes over one kan_server_step, as allocated. Any pointer may be NULL. */
int kan_server_status(const kan_server* server, size_t* waiting, size_t* active,
                      size_t* finished, size_t* hbm_in_use, size_t* hbm_peak,
                      size_t* hbm_measured_peak);

#ifdef __cplusplus
}
#endif
#endif
