// bfs_multi.h -- device-side types of the multi-source (lane-mask) search,
// shared by its persistent driver and the server's stepped driver.
#pragma once

#include "bfs_common.cuh"

namespace bfsk {

struct MTask {
    long long start;
    int len;
    int v;        // index of the row's first chunk task: its lane mask is hubmask[v]
};

// Control block of a multi-source launch / server slot.
struct MCtrl {
    BarrierState b;
    unsigned long long accn[3];    // vertices that gained lane bits (new union frontier size)
    unsigned long long accm[3];    // their degree sum
    unsigned long long mdone[3];   // degree of vertices every active lane has now seen
    unsigned long long ntask[3];   // top-down chunk tasks
    unsigned long long found[3];   // lanes that found at least one vertex
    long long iterations;
    // server slot state carried across launches (bfs_serve_kernel)
    long long s_done;              // iterations run by the last launch
    unsigned long long s_finished; // lanes whose search ended in the last launch
    long long s_nf, s_mf;          // union frontier size / degree sum after the last level
    int s_dir;                     // direction of the last level
    int s_qsel;                    // which queue holds the frontier
    unsigned long long qlen[2];    // lengths of the two vertex queues (frontier / touched)
    __host__ __device__ void zero_slot(int s) {
        accn[s] = 0;
        accm[s] = 0;
        mdone[s] = 0;
        ntask[s] = 0;
        found[s] = 0;
    }
};

// Per-lane table in device memory: output rows, start iteration, root.
struct LaneTable {
    int* rows[64];
    int* prow[64];
    int start[64];
    int roots[64];
};

struct MultiParams {
    const long long* __restrict__ off;
    const int* __restrict__ cols;
    const int* __restrict__ cols_bu;   // rows as the bottom-up pulls scan them (cols, or hub-first)
    long long n, nnz;
    unsigned long long* seen;
    unsigned long long* front;
    unsigned long long* next;
    MCtrl* ctrl;
    MTask* tasks;
    unsigned long long* hubmask;   // [task_cap] lane masks of chunked rows
    long long task_cap;
    int* q0;                       // vertex queues, n + 64 entries each
    int* q1;
    int* const* rows;
    const int* start;
    const int* roots;
    unsigned long long active;
    int mode, alpha, beta, big_deg;
    unsigned long long timeout_ns;
    unsigned expected;
};

}  // namespace bfsk
