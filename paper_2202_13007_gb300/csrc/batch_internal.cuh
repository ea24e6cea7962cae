// batch_internal.cuh -- work-list format of the persistent batch kernel,
// shared by the batch planner and the request server.
#pragma once

#include <vector>

#include "blaz_internal.cuh"

namespace blaz {
namespace batch {

struct DevOp {
    int32_t kind;
    int32_t vec;          // COMPRESS: 16-byte vector loads allowed
    int64_t nbc;          // blocks per block-row of the block loop's matrix
    const double *fa, *sa;
    const uint8_t *pa;
    const int8_t *ca;
    const double *fb, *sb;
    const uint8_t *pb;
    const int8_t *cb;
    double *fo, *so;
    uint8_t *po;
    int8_t *co;
    const double *A;
    int64_t lda;
    double c;
    double *result;
    const double *B;
    int64_t ldb, m;
    double *C;
    int64_t ldc;
    double *scratch;      // MATMUL: decompressed a (n x k, leading dimension k)
    int64_t n, k;
    int32_t first_item;   // first block item of the op
    int32_t nitems;       // number of block items of the op
    int64_t partial_base; // DOT: first slot of the op in partials[]
};

struct Item {
    int32_t op;
    int32_t tile;   // 0: blocks [b0, b1); 1: product tile at rows b0, columns b1
    int64_t b0, b1;
};

// Host: descriptors and work items of `ops` (validated) for `blocks_per_item`;
// the decompressed operands of the products live at scratch + scratch_off[i]
// (scratch may be null while sizing: pass scratch_bytes_out to learn the size).
void build_work(const blaz_op *ops, int nops, int64_t blocks_per_item, char *scratch, std::vector<DevOp> &dops,
                std::vector<Item> &items, int64_t &partials, size_t &scratch_bytes_out, int &ngemm);
// Validation of one operation (shapes, pointers, leading dimensions).
int check_op(const blaz_op &o);
// Device: the persistent kernel; counters = [next item, done per op] (zeroed).
int launch(const DevOp *d_ops, const Item *d_items, int nitems, unsigned *d_counters, double *d_partials, int grid,
           cudaStream_t st);

}  // namespace batch
}  // namespace blaz
