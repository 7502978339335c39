/*
 * pt_probes.h -- measurement probes of libpathrecycle.so: the memory rates
 * that bound the recycled passes, measured on the device they run on.
 *
 * The paper has no counterpart: these calls exist to give the passes a
 * roofline.  The recycled forward pass gathers 4-byte extinction values
 * along shadow rays (L2-resident grids), the gradient pass adds FP64 terms
 * into a voxel grid with reductions that are resolved in L2, and both
 * stream stored records from HBM.  Each probe runs one of those access
 * patterns alone, as fast as the device allows, so that a pass's achieved
 * rate can be divided by it.
 *
 * Conventions as in pathrecycle.h (device pointers of the current device,
 * caller-owned; asynchronous on `stream`; status return, pt_last_error()).
 */
#ifndef PT_PROBES_H
#define PT_PROBES_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* access patterns (`kind`) */
enum {
    PT_PROBE_GATHER_F32 = 0,   /* 4-byte loads at uniformly random indices of buf (float32[n])      */
    PT_PROBE_RED_F64 = 1,      /* FP64 reductions (add, result unused) at random indices (double[n]) */
    PT_PROBE_RED_F64_WARP = 2, /* FP64 reductions, the 32 lanes of a warp on 32 consecutive doubles  */
    PT_PROBE_RED_F64_SAME = 3, /* FP64 reductions, the 32 lanes of a warp on one random address     */
    PT_PROBE_RED_F32 = 4,      /* FP32 reductions at random indices (float32[n])                     */
    PT_PROBE_COPY = 5,         /* streaming copy src -> buf of n 16-byte elements (HBM when large)   */
    PT_PROBE_SHARED_F32 = 6,   /* FP32 atomic adds into a 4096-entry shared-memory table, random slots */
    PT_PROBE_SHARED_F32_RUN4 = 7, /* the same, lanes in groups of 4 on one slot                       */
    PT_PROBE_SHARED_U32 = 8,   /* 32-bit integer atomic adds, random slots                          */
    PT_PROBE_SHARED_F64 = 9,   /* FP64 atomic adds into a 2048-entry shared table, random slots      */
    PT_PROBE_KINDS = 10
};

/*
 * Runs one probe: `blocks` blocks of 256 threads; for the random kinds every
 * thread performs `iters` accesses (indices from a per-thread linear
 * congruential sequence, so accesses are independent of loaded values);
 * PT_PROBE_COPY copies all n elements once (grid-stride; `iters` unused).
 *   buf   device buffer: float32[n] (GATHER, RED_F32), double[n] (RED_F64*),
 *         16-byte elements[n] (COPY destination), float32[blocks * 256]
 *         (SHARED_*: each thread writes one value read back from its
 *         block's table, so the adds are not optimised away).  The
 *         reduction probes add into it (its values change); the gather
 *         probe only reads it.
 *   n     elements of buf; a power of two >= 32 for the random kinds
 *         (SHARED_*: at least blocks * 256).
 *   src   COPY only: the source, 16-byte elements[n]; NULL otherwise.
 *   sink  GATHER only: float32[blocks * 256], one sum per thread (keeps the
 *         loads from being optimised away); NULL otherwise.
 * Accesses stay inside buf by construction (indices masked to n - 1).
 * Errors: PT_E_INVALID for a null buffer, n not a power of two, blocks or
 * iters out of range (blocks in 1..2^20, iters in 1..2^24); PT_E_CUDA if the
 * launch fails.
 */
int pt_probe(int kind, void* buf, int64_t n, const void* src, int64_t iters, int blocks, float* sink,
             void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PT_PROBES_H */
