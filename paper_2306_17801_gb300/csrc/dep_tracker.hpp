// Dependency tracker behind intent marking (Sec. 3.1.2).
//
// For every object ID it keeps the last write and the reads since that write,
// each as (context, launch sequence number).  Before a launch that accesses
// an object, begin() asks the backend to make the launching context wait for
// exactly the conflicting accesses made on other contexts:
//   read  -> the last write;
//   write -> the last write and every read since it.
// Accesses on the same context are already in program order, and reads are
// never ordered among themselves (the strong write-ordering rule stated at
// the end of Sec. 3.1.2).  A wait is elided when the waiter is already known
// to wait for that launch (or a later one of the same context), or when the
// backend reports the launch finished.
//
// The tracker is pure host logic, parameterised on a backend so that the same
// code drives CUDA events in the library and a recording fake in the
// host-only simulator.  Backend interface:
//   bool complete(uint64_t ctx, uint64_t seq);              // non-blocking query
//   void wait(uint64_t waiter, uint64_t ctx, uint64_t seq); // enqueue a wait
//   void elided(uint64_t waiter, uint64_t ctx, uint64_t seq);
// The caller serialises access (one mutex around the tracker).
#pragma once

#include <cstdint>
#include <unordered_map>
#include <vector>

namespace apcg {

enum : int { kRead = 1, kWrite = 2, kReadWrite = 3 };

struct Access {
  uint64_t ctx;
  uint64_t seq;
};

struct ObjRecord {
  bool has_writer = false;
  Access writer{0, 0};
  std::vector<Access> readers;  // at most one entry per context: its latest read
};

class DepTracker {
 public:
  // Accesses that a `mode` access to `id` must be ordered after.
  std::vector<Access> conflicts(uint64_t id, int mode) const {
    std::vector<Access> out;
    auto it = objs_.find(id);
    if (it == objs_.end()) return out;
    const ObjRecord& o = it->second;
    if (o.has_writer) out.push_back(o.writer);
    if (mode & kWrite)
      for (const Access& a : o.readers) out.push_back(a);
    return out;
  }

  template <class Backend>
  void begin(Backend& be, uint64_t ctx, uint64_t id, int mode) {
    for (const Access& a : conflicts(id, mode)) {
      if (a.ctx == ctx) continue;  // program order on one context
      uint64_t& k = known_[ctx][a.ctx];
      if (k >= a.seq || be.complete(a.ctx, a.seq)) {
        be.elided(ctx, a.ctx, a.seq);
        if (k < a.seq) k = a.seq;
        continue;
      }
      be.wait(ctx, a.ctx, a.seq);
      k = a.seq;
    }
  }

  void end(uint64_t ctx, uint64_t id, int mode, uint64_t seq) {
    ObjRecord& o = objs_[id];
    if (mode & kWrite) {
      o.has_writer = true;
      o.writer = Access{ctx, seq};
      o.readers.clear();
      return;
    }
    for (Access& a : o.readers)
      if (a.ctx == ctx) {
        if (seq > a.seq) a.seq = seq;
        return;
      }
    o.readers.push_back(Access{ctx, seq});
  }

  // A context that waited for all work of `waitee` up to `seq` (an explicit
  // context-to-context wait) knows about it.
  void note_known(uint64_t waiter, uint64_t waitee, uint64_t seq) {
    uint64_t& k = known_[waiter][waitee];
    if (k < seq) k = seq;
  }

  void forget(uint64_t id) { objs_.erase(id); }

  void forget_context(uint64_t ctx) { known_.erase(ctx); }

 private:
  std::unordered_map<uint64_t, ObjRecord> objs_;
  std::unordered_map<uint64_t, std::unordered_map<uint64_t, uint64_t>> known_;
};

}  // namespace apcg
