// ws_multi.cuh -- persistent launches over many tables (batched plans, the
// serving loop, the no-allocation call).
//
// A phase is a list of items (table, op kind, op arrays).  The host cuts every
// item into chunks of kMultiChunk ops and groups them by the item's table
// configuration -- one entry of a fixed menu of compiled (scheme, metadata,
// bucket slots, tile) combinations -- and op kind.  One persistent kernel per
// group takes the group's chunks from a ticket counter (dynamic scheduling:
// item sizes differ by four orders of magnitude); each warp serves a 256-op
// share of a chunk with the lane and tile code of the single-table kernel.
// A group's chunks come from an explicit list, or from prefix sums of the
// chunk counts of a range of items (the no-allocation call, whose scratch has
// a fixed size).  Each (menu entry, kind) is its own kernel in its own
// translation unit (ws_multi_<entry>.cu), compiled in parallel.
#pragma once
#include "ws_kernels.cuh"

namespace ws {

constexpr int kWarpShare = 256;                   // ops of a chunk per warp
constexpr int kMultiChunk = kWarps * kWarpShare;  // ops per chunk = one block iteration

struct MultiItem {
  TableView tv;
  BatchArgs a;
  int kind;      // KIND_QUERY / KIND_UPSERT / KIND_ERASE / KIND_MIXED (per-op codes in a.ops)
  int cfg;       // index into the menu
  int lockfree;  // no erase of this table in this phase
  int pad;
};

struct MultiChunk {
  u32 item;
  u32 pad;
  u64 start;
};

// One group's work: chunks [0, n_chunks) from the list `chunks`, or -- with
// chunks null -- chunk c is chunk c - prefix[item] of the item with
// prefix[item] <= prefix[i0] + c < prefix[item + 1], item in [i0, i1).
struct MultiGroup {
  const MultiItem* items;
  const MultiChunk* chunks;
  const u32* prefix;
  u32 i0, i1;
  u32 n_chunks;
  u32* ticket;  // zeroed before the launch
};

// Menu of compiled configurations (scheme, metadata, bucket slots, tile).
#define WS_MULTI_MENU(X)            \
  X(0, SCHEME_DOUBLE, false, 8, 4)  \
  X(1, SCHEME_DOUBLE, false, 8, 8)  \
  X(2, SCHEME_DOUBLE, true, 32, 4)  \
  X(3, SCHEME_DOUBLE, true, 32, 8)  \
  X(4, SCHEME_P2, false, 32, 8)     \
  X(5, SCHEME_P2, false, 32, 32)    \
  X(6, SCHEME_P2, true, 32, 4)      \
  X(7, SCHEME_P2, true, 32, 8)
constexpr int kMultiMenu = 8;

// Menu index of a configuration, or -1.
inline int multi_menu_index(int scheme, bool meta, int B, int T) {
#define WS_MULTI_FIND(ID, SCH, MT, BB, TT) \
  if (scheme == SCH && meta == MT && B == BB && T == TT) return ID;
  WS_MULTI_MENU(WS_MULTI_FIND)
#undef WS_MULTI_FIND
  return -1;
}

// Runs group g on stream s with the kernel of menu entry `cfg` and op kind
// `kind` (grid: resident blocks of all SMs, at most one block per chunk).
cudaError_t launch_multi(int cfg, int kind, const MultiGroup& g, cudaStream_t s, int num_sms);

}  // namespace ws
