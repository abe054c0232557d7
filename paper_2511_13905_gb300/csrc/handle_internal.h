// handle_internal.h -- entry points shared by api.cu, serve.cu and tune.cu that are not part
// of the public C ABI: a step report read without synchronising the handle's stream, and
// the table of tuned cluster-engine block shares.
#pragma once

#include "../../include/pgdto.h"

// The report of a handle's last launch as the device wrote it: pgdto_info plus the four
// words of the grid control block that carry a sticky error and the abort flag.
struct pgdto_info_slot {
    pgdto_info info;
    int ctrl[4];
};

// Enqueue the copy of the handle's report into `slot` (pinned host memory) on the handle's
// stream, behind the launch it reports on.  Returns without waiting.
pgdto_status pgdto_info_enqueue(pgdto_handle* h, pgdto_info_slot* slot);

// Interpret a slot whose copy has completed (the caller waited on an event recorded after
// pgdto_info_enqueue): the step's status, and `info` when non-null.  An error clears the
// control block with an asynchronous memset on the handle's stream, as pgdto_last_info does.
pgdto_status pgdto_info_collect(pgdto_handle* h, const pgdto_info_slot* slot, pgdto_info* info);

// 1 when the handle's steps run on the grid engine (every SM on the one problem), 0 when
// they run on one thread-block cluster; the server batches only the latter.
int pgdto_handle_whole_gpu(const pgdto_handle* h);

// The cluster-engine block share pgdto_autotune_batch chose for problems of n variables on
// `device` (the table is kept per power-of-two bucket of n), or 0 when none was chosen.
int pgdto_tuned_cluster_elems(int device, int64_t n);
void pgdto_set_tuned_cluster_elems(int device, int64_t n, int elems);
