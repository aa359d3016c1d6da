// Device tensors, a bump arena and the reverse-mode tape of the engine.
#pragma once
#include <functional>
#include <initializer_list>
#include <string>
#include <vector>

#include "common.h"

namespace sctm {

// A strided view of device memory.  `grad` (if not null) points at the gradient
// buffer laid out exactly like `data`, so every view transform keeps the two
// aligned and adjoints can be accumulated through views.
struct Tensor {
  double* data = nullptr;
  double* grad = nullptr;
  int nd = 0;
  int shape[kMaxDims] = {0};
  long long stride[kMaxDims] = {0};

  long long numel() const {
    long long t = 1;
    for (int i = 0; i < nd; ++i) t *= shape[i];
    return t;
  }
  bool contiguous() const {
    long long s = 1;
    for (int i = nd - 1; i >= 0; --i) {
      if (shape[i] != 1 && stride[i] != s) return false;
      s *= shape[i];
    }
    return true;
  }
  // reorder dims: new dim i = old dim p[i]
  Tensor perm(std::initializer_list<int> p) const {
    Tensor t = *this;
    int i = 0;
    for (int d : p) {
      t.shape[i] = shape[d];
      t.stride[i] = stride[d];
      ++i;
    }
    return t;
  }
  Tensor rev() const {  // reverse dim order (transpose of a matrix)
    Tensor t = *this;
    for (int i = 0; i < nd; ++i) {
      t.shape[i] = shape[nd - 1 - i];
      t.stride[i] = stride[nd - 1 - i];
    }
    return t;
  }
  Tensor reshape(std::initializer_list<int> s) const;   // contiguous only
  Tensor sub(int dim, int index) const {                 // drop one dim at an index
    Tensor t;
    t.data = data + index * stride[dim];
    t.grad = grad ? grad + index * stride[dim] : nullptr;
    t.nd = nd - 1;
    for (int i = 0, j = 0; i < nd; ++i) {
      if (i == dim) continue;
      t.shape[j] = shape[i];
      t.stride[j] = stride[i];
      ++j;
    }
    return t;
  }
};

// Bump allocator over one device allocation.  Forward intermediates of a taped
// region live until the region's reverse pass is done; mark/release frees them.
// A second stack grows down from the top end (alloc_high): it holds data that
// the forward pass leaves for the reverse pass, which consumes it last in,
// first out.
class Arena {
 public:
  Arena() = default;
  ~Arena();
  void reserve(size_t bytes);
  double* alloc(long long n);          // 256-byte aligned, uninitialised
  double* alloc_high(long long n);     // from the top end, 256-byte aligned, uninitialised
  size_t mark() const { return top_; }
  void release(size_t m) { top_ = m; }
  size_t mark_high() const { return hi_; }
  void release_high(size_t m) { hi_ = m; }
  size_t capacity() const { return cap_; }
  size_t high_water() const { return high_; }

 private:
  char* base_ = nullptr;
  size_t cap_ = 0, top_ = 0, hi_ = 0, high_ = 0;
};

struct Tape {
  bool active = false;
  std::vector<std::function<void()>> ops;
  void push(std::function<void()> f) {
    if (active) ops.push_back(std::move(f));
  }
  void backward() { backward_from(0); }
  // run (in reverse) and drop only the closures recorded after mark()
  size_t mark() const { return ops.size(); }
  void backward_from(size_t m) {
    for (size_t i = ops.size(); i > m; --i) ops[i - 1]();
    ops.resize(m);
  }
};

}  // namespace sctm
