/* hweno_checked.h -- entry points exported by libhweno_checked.so only: the
 * library built with -DHWENO_CHECKED, in which the stage kernels test their
 * shared- and global-memory indices against the buffers' extents.  A bad
 * index is counted, the first one is recorded and the access is skipped (a
 * load gives 0); nothing traps, so the CUDA context stays usable.  The paper
 * has no counterpart: this is a development aid standing in for a memory
 * checker.  Every other entry point of include/hweno.h is exported too, with
 * the same meaning.
 *
 * Each compiled unit keeps its own check word: the 2D stage kernels
 * (hweno_check_stage2d), the 1D stage kernels (hweno_check_stage1d) and the
 * self-test (hweno_check_probe).
 */
#ifndef HWENO_CHECKED_H
#define HWENO_CHECKED_H

#ifdef __cplusplus
extern "C" {
#endif

/* Copy the unit's check word into out4 (host array of 4): [0] number of
 * accesses skipped since the last reset, [1] the first one's site number,
 * [2] its index, [3] the extent it was tested against (low 32 bits).  With
 * reset != 0 the word is cleared afterwards.  Returns a cudaError_t value
 * (0 = success).  Synchronises with the device. */
int hweno_check_stage2d(unsigned int* out4, int reset);
int hweno_check_stage1d(unsigned int* out4, int reset);
int hweno_check_probe(unsigned int* out4, int reset);

/* Runs the index test on one index inside its extent and one outside,
 * accessing no memory at either; pass_out (host array of 2) receives 1, 0
 * and hweno_check_probe then reports one skipped access at site 99, index 7,
 * extent 5.  Returns a cudaError_t value. */
int hweno_check_selftest(int* pass_out);

#ifdef __cplusplus
}
#endif

#endif
