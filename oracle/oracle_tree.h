/*
 * oracle_tree.h -- the oracle's tree and list record, shared by the oracle's
 * own translation units (the Laplace and Helmholtz FMMs walk the same tree).
 * TEST INFRASTRUCTURE ONLY; never included by the GPU library.
 */
#ifndef ORACLE_TREE_H
#define ORACLE_TREE_H
#include <stdint.h>

typedef struct {
  int32_t *a;
  int64_t n, cap;
} ivec;

struct oracle_tree {
  int64_t n;
  double lo[3], D;
  int leaf_size, max_depth;
  uint64_t *keys;    /* sorted */
  int32_t *perm;     /* perm[i] = input index of the i-th sorted point */
  double *xyz;       /* sorted coordinates */
  int nlevels;
  int32_t *level_offset;
  int64_t nboxes;
  uint64_t *box_key; /* anchor key at the box's level */
  int32_t *box_level, *box_first, *box_count, *box_parent, *box_child, *box_nchild;
  int32_t (*anchor)[3];
  double (*center)[3];
  double *side; /* per level */
  ivec *U, *V, *W, *X; /* per box */
};

#endif
