// Level layout (host): oct neighbour table and interface-face records.
//
// A level is a list of octs (Sect. 3.3: the restriction works on octs, the
// 2^ndim children of a cell).  For the device the level needs, per oct, the
// index of the six face-neighbour octs (or -1 where the level ends: a coarser
// leaf or a physical wall), and, for octs that carry interface descriptors,
// a record mapping (cell, direction) to the descriptor.
#include <cstring>
#include <string>
#include <vector>

#include "ats_internal.h"

namespace ats {
namespace {

// Open-addressing hash of packed oct coordinates -> oct index.
class OctHash {
 public:
  explicit OctHash(int64_t n) {
    size_t cap = 16;
    while (cap < (size_t)n * 2 + 16) cap <<= 1;
    keys_.assign(cap, kEmpty);
    vals_.assign(cap, -1);
    mask_ = cap - 1;
  }
  static uint64_t pack(int64_t x, int64_t y, int64_t z) {
    const int64_t off = int64_t(1) << 20;
    return (uint64_t(x + off) << 42) | (uint64_t(y + off) << 21) | uint64_t(z + off);
  }
  // returns false if the key was already present
  bool insert(uint64_t k, int32_t v) {
    size_t h = mix(k) & mask_;
    while (keys_[h] != kEmpty) {
      if (keys_[h] == k) return false;
      h = (h + 1) & mask_;
    }
    keys_[h] = k;
    vals_[h] = v;
    return true;
  }
  int32_t find(uint64_t k) const {
    size_t h = mix(k) & mask_;
    while (keys_[h] != kEmpty) {
      if (keys_[h] == k) return vals_[h];
      h = (h + 1) & mask_;
    }
    return -1;
  }

 private:
  static constexpr uint64_t kEmpty = ~uint64_t(0);
  static uint64_t mix(uint64_t k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdULL;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ULL;
    k ^= k >> 33;
    return k;
  }
  std::vector<uint64_t> keys_;
  std::vector<int32_t> vals_;
  size_t mask_ = 0;
};

constexpr int kAxis[6] = {0, 0, 1, 1, 2, 2};
constexpr int kSign[6] = {-1, 1, -1, 1, -1, 1};

}  // namespace

std::string build_layout(const ats_level_desc &d, Layout &out) {
  if (d.n_oct <= 0) return "level has no octs";
  if (d.n_oct > (int64_t(1) << 28)) return "level too large (n_oct > 2^28)";
  if (!d.oct_xyz) return "oct_xyz is NULL";
  if (!(d.dx > 0.0)) return "dx must be > 0";
  if (d.n_face < 0 || (d.n_face > 0 && (!d.face_cell || !d.face_dir || !d.face_kind || !d.face_rel)))
    return "face arrays missing";
  const int64_t n = d.n_oct;
  const int64_t N = 8 * n;
  out.n_oct = n;
  OctHash hash(n);
  for (int64_t o = 0; o < n; ++o) {
    const int32_t *c = d.oct_xyz + 3 * o;
    for (int k = 0; k < 3; ++k)
      if (c[k] <= -(1 << 20) + 2 || c[k] >= (1 << 20) - 2) return "oct coordinate out of range";
    if (!hash.insert(OctHash::pack(c[0], c[1], c[2]), (int32_t)o)) return "duplicate oct";
  }
  out.nbr.assign(6 * n, -1);
  for (int64_t o = 0; o < n; ++o) {
    const int32_t *c = d.oct_xyz + 3 * o;
    for (int dir = 0; dir < 6; ++dir) {
      int64_t q[3] = {c[0], c[1], c[2]};
      q[kAxis[dir]] += kSign[dir];
      out.nbr[6 * o + dir] = hash.find(OctHash::pack(q[0], q[1], q[2]));
    }
  }
  auto is_leaf = [&](int64_t cell) -> bool {
    if (!d.leaf_mask) return true;
    return (d.leaf_mask[cell >> 3] >> (cell & 7)) & 1;
  };
  // the neighbour cell of (cell, dir) inside this level, or -1
  auto nb_cell = [&](int64_t cell, int dir) -> int64_t {
    const int64_t o = cell >> 3;
    const int c = (int)(cell & 7);
    const int a = kAxis[dir];
    const int bit = (c >> a) & 1;
    const bool inside = (kSign[dir] > 0) ? (bit == 0) : (bit == 1);
    if (inside) return 8 * o + (c ^ (1 << a));
    const int32_t no = out.nbr[6 * o + dir];
    if (no < 0) return -1;
    return 8 * (int64_t)no + (c ^ (1 << a));
  };

  // validate descriptors and build the per-oct face records
  out.frec.assign(n, -1);
  out.rec_face.clear();
  out.n_rec = 0;
  for (int64_t f = 0; f < d.n_face; ++f) {
    const int64_t cell = d.face_cell[f];
    const int dir = d.face_dir[f];
    if (cell < 0 || cell >= N) return "face_cell out of range";
    if (dir < 0 || dir > 5) return "face_dir out of range";
    if (d.face_kind[f] < 0 || d.face_kind[f] > 2) return "bad face_kind";
    if (d.face_rel[f] < 0 || d.face_rel[f] > 2) return "bad face_rel";
    if (d.face_alpha) {
      const double al = d.face_alpha[f];
      if (!(al >= 0.0 && al <= 1.0)) return "face_alpha outside [0,1]";
    }
    if (!is_leaf(cell)) return "descriptor on a non-leaf cell";
    const int64_t j = nb_cell(cell, dir);
    if (j >= 0 && is_leaf(j)) return "descriptor on an interior face";
    const int64_t o = cell >> 3;
    if (out.frec[o] < 0) {
      out.frec[o] = (int32_t)out.n_rec++;
      out.rec_face.resize(out.n_rec * 48, -1);
    }
    int32_t &slot = out.rec_face[out.frec[o] * 48 + (cell & 7) * 6 + dir];
    if (slot >= 0) return "duplicate face descriptor";
    slot = (int32_t)f;
  }
  return std::string();
}

}  // namespace ats
