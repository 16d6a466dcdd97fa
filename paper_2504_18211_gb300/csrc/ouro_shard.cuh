/* Build sharding of the kernel files.
 *
 * Every kernel of the allocator is a template over the queue form (the six
 * forms of Sec. 3), and compiling all six in one object takes minutes.  The
 * build therefore compiles each kernel file seven times:
 *   -DOURO_SHARD=-1   the host entry points and the form-independent
 *                     kernels; the per-form launchers are only declared;
 *   -DOURO_SHARD=v    the per-form launchers (and so the kernels) of form v
 *                     only, no entry points.
 * Without OURO_SHARD a kernel file is one ordinary object holding all of it.
 *
 * A per-form launcher is a function template `template <int V> ouro_status
 * f(...)` of external linkage whose signature names no type of the file's
 * anonymous namespace.  After its definition the file states
 *   #define INST_F(PRE, V) PRE template ouro_status f<V>(...);
 *   OURO_SHARD_INSTANTIATE(INST_F)
 * which expands to nothing (implicit instantiation), to an `extern template`
 * declaration of all six forms (entries object), or to the explicit
 * instantiation of the one form the object compiles.
 */
#ifndef OURO_SHARD_CUH
#define OURO_SHARD_CUH

#include "ouro.h"

#if defined(OURO_SHARD) && OURO_SHARD >= 0
#define OURO_SHARD_ENTRIES 0   /* a per-form object: no entry points */
#else
#define OURO_SHARD_ENTRIES 1
#endif

#define OURO_SHARD_EACH(M, PRE)    \
  M(PRE, OURO_PAGE_ARRAY)          \
  M(PRE, OURO_PAGE_VLIST)          \
  M(PRE, OURO_CHUNK_ARRAY)         \
  M(PRE, OURO_CHUNK_VLIST)         \
  M(PRE, OURO_PAGE_VARRAY)         \
  M(PRE, OURO_CHUNK_VARRAY)

#if !defined(OURO_SHARD)
#define OURO_SHARD_INSTANTIATE(M)
#elif OURO_SHARD < 0
#define OURO_SHARD_INSTANTIATE(M) OURO_SHARD_EACH(M, extern)
#else
#define OURO_SHARD_INSTANTIATE(M) M(, OURO_SHARD)
#endif

#endif
