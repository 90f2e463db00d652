// Index persistence: sofa_save writes every array of a built index (and a
// trained proposal network) to one file; sofa_load recreates the handle on the
// current device from it, without the raw data or any of the build's work.
//
// File: the 8-byte magic "SOFAIDX3", a fixed header of 64-bit fields, the
// size of the build's key-sorted run (rows beyond it are the appended region
// of sofa_insert; a "SOFAIDX2" file has no such field and no region), then one
// section per array -- a 64-bit byte count followed by the bytes, in a fixed
// order (optional arrays have count 0 when absent) -- then the proposal
// network.  Arrays move between device and file through a pinned staging
// buffer in 64 MiB pieces.
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "sofa_internal.cuh"

namespace sofa {

void set_error(const std::string& msg);

namespace {

constexpr char MAGIC[8] = {'S', 'O', 'F', 'A', 'I', 'D', 'X', '3'};
constexpr char MAGIC_V2[8] = {'S', 'O', 'F', 'A', 'I', 'D', 'X', '2'};
constexpr size_t PIECE = (size_t)64 << 20;

struct Header {
  int64_t N, n, l, alpha, LW, nsel, NB, bps, nyq_first, leaf_tiles, T, L, precision, keybits, has_mlp;
  double delta_d, delta_q, vmax, outer;
};

struct Staging {
  void* p = nullptr;
  ~Staging() {
    if (p) cudaFreeHost(p);
  }
  int get() {
    if (!p && cudaMallocHost(&p, PIECE) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      return fail(SOFA_ERR_OOM, "pinned staging buffer allocation failed");
    }
    return 0;
  }
};

int write_array(FILE* f, Staging& sg, const void* dev, size_t bytes) {
  const uint64_t b = dev ? bytes : 0;
  if (fwrite(&b, sizeof(b), 1, f) != 1) return fail(SOFA_ERR_INVALID_ARG, "write failed");
  if (!b) return 0;
  if (int rc = sg.get()) return rc;
  for (size_t off = 0; off < b; off += PIECE) {
    const size_t m = b - off < PIECE ? b - off : PIECE;
    SOFA_CUDA(cudaMemcpy(sg.p, static_cast<const char*>(dev) + off, m, cudaMemcpyDeviceToHost));
    if (fwrite(sg.p, 1, m, f) != m) return fail(SOFA_ERR_INVALID_ARG, "write failed");
  }
  return 0;
}

// Reads a section of exactly `bytes` bytes (or an empty one when `optional`)
// into a new device allocation.
template <typename T>
int read_array(FILE* f, Staging& sg, T** dev, size_t bytes, bool optional, int64_t* acct) {
  uint64_t b = 0;
  if (fread(&b, sizeof(b), 1, f) != 1) return fail(SOFA_ERR_INVALID_ARG, "truncated index file");
  if (b == 0 && optional) return 0;
  if (b != bytes) return fail(SOFA_ERR_INVALID_ARG, "index file section has an unexpected size");
  if (dev_malloc((void**)dev, b) != cudaSuccess) {
    cudaGetLastError();
    return fail(SOFA_ERR_OOM, "device allocation failed while loading an index");
  }
  *acct += (int64_t)b;
  if (int rc = sg.get()) return rc;
  for (size_t off = 0; off < b; off += PIECE) {
    const size_t m = b - off < PIECE ? b - off : PIECE;
    if (fread(sg.p, 1, m, f) != m) return fail(SOFA_ERR_INVALID_ARG, "truncated index file");
    SOFA_CUDA(cudaMemcpy(reinterpret_cast<char*>(*dev) + off, sg.p, m, cudaMemcpyHostToDevice));
  }
  return 0;
}

struct Sizes {
  size_t nsel_i, nsel_d, basis, beta, tab, words, Z, N4, N8, keyorder, tenv, lenv, Z8, VC, vsr, vw, Zh;
};

Sizes sizes_of(const Index* ix) {
  Sizes z;
  const size_t N = (size_t)ix->N;
  z.nsel_i = (size_t)ix->nsel * sizeof(int32_t);
  z.nsel_d = (size_t)ix->nsel * sizeof(double);
  z.basis = (size_t)ix->n * ix->NB * sizeof(float);
  z.beta = (size_t)ix->LW * (ix->alpha + 1) * sizeof(float);
  z.tab = (size_t)ix->LW * MAX_ALPHA * sizeof(float2);
  z.words = N * ix->LW;
  z.Z = N * ix->n * sizeof(float);
  z.N4 = N * 4;
  z.N8 = N * 8;
  z.keyorder = 64;
  z.tenv = (size_t)ix->T * 2 * ix->LW;
  z.lenv = (size_t)ix->L * 2 * ix->LW;
  z.Z8 = N * ix->n;
  z.VC = N * ix->NB;
  z.vsr = N * sizeof(float2);
  z.vw = (size_t)ix->NB * sizeof(float);
  z.Zh = N * ix->n * sizeof(__half);
  return z;
}

int save_index(const Index* ix, FILE* f) {
  Header h;
  std::memset(&h, 0, sizeof(h));
  h.N = ix->N;
  h.n = ix->n;
  h.l = ix->l;
  h.alpha = ix->alpha;
  h.LW = ix->LW;
  h.nsel = ix->nsel;
  h.NB = ix->NB;
  h.bps = ix->bps;
  h.nyq_first = ix->nyq_first;
  h.leaf_tiles = ix->leaf_tiles;
  h.T = ix->T;
  h.L = ix->L;
  h.precision = ix->precision;
  h.keybits = ix->keybits;
  h.delta_d = ix->delta_d;
  h.delta_q = ix->delta_q;
  h.vmax = ix->vmax;
  h.outer = ix->outer;
  h.has_mlp = ix->mlp ? 1 : 0;
  const int64_t Ns = ix->Ns;
  if (fwrite(MAGIC, 1, 8, f) != 8 || fwrite(&h, sizeof(h), 1, f) != 1 || fwrite(&Ns, sizeof(Ns), 1, f) != 1)
    return fail(SOFA_ERR_INVALID_ARG, "write failed");
  const Sizes z = sizes_of(ix);
  Staging sg;
  const struct {
    const void* p;
    size_t b;
  } arrays[] = {{ix->sel, z.nsel_i},   {ix->sel_k, z.nsel_i}, {ix->sel_part, z.nsel_i}, {ix->var, z.nsel_d},
                {ix->basis, z.basis},   {ix->beta, z.beta},    {ix->edge, z.tab},         {ix->ch, z.tab},
                {ix->ch16, z.tab / 2},  {ix->words, z.words},  {ix->Z, z.Z},              {ix->perm, z.N4},
                {ix->keys, z.N8},       {ix->keyorder, z.keyorder}, {ix->tenv, z.tenv},   {ix->lenv, z.lenv},
                {ix->xn, z.N4},         {ix->Z8, z.Z8},        {ix->s8, z.N4},            {ix->e8, z.N4},
                {ix->VC, z.VC},         {ix->vsr, z.vsr},      {ix->vw, z.vw},            {ix->Zh, z.Zh}};
  for (const auto& a : arrays)
    if (int rc = write_array(f, sg, a.p, a.b)) return rc;
  if (ix->mlp)
    if (int rc = mlp_save(ix, f)) return rc;
  return 0;
}

int load_index(Index* ix, FILE* f, cudaStream_t st) {
  char magic[8];
  Header h;
  if (fread(magic, 1, 8, f) != 8) return fail(SOFA_ERR_INVALID_ARG, "not an index file");
  const bool v3 = std::memcmp(magic, MAGIC, 8) == 0;
  if (!v3 && std::memcmp(magic, MAGIC_V2, 8) != 0) return fail(SOFA_ERR_INVALID_ARG, "not an index file");
  if (fread(&h, sizeof(h), 1, f) != 1) return fail(SOFA_ERR_INVALID_ARG, "truncated index file");
  int64_t Ns = h.N;
  if (v3 && fread(&Ns, sizeof(Ns), 1, f) != 1) return fail(SOFA_ERR_INVALID_ARG, "truncated index file");
  if (Ns < 1 || Ns > h.N) return fail(SOFA_ERR_INVALID_ARG, "index file header is inconsistent");
  if (h.N < 1 || h.N >= ((int64_t)1 << 31) || h.n < 4 || h.n > 1024 || (h.LW != 16 && h.LW != 32) ||
      h.NB != 2 * h.LW || h.nsel < 1 || h.nsel > 2 * h.LW || h.alpha < 2 || h.alpha > 256 || h.keybits < 0 ||
      h.keybits > 64 || h.leaf_tiles < 1 || h.leaf_tiles > 256 || h.T != ceil_div(h.N, TILE) ||
      h.L != ceil_div(h.T, h.leaf_tiles))
    return fail(SOFA_ERR_INVALID_ARG, "index file header is inconsistent");
  ix->N = h.N;
  ix->Ns = Ns;
  ix->n = (int)h.n;
  ix->l = (int)h.l;
  ix->alpha = (int)h.alpha;
  ix->LW = (int)h.LW;
  ix->nsel = (int)h.nsel;
  ix->NB = (int)h.NB;
  ix->bps = (int)h.bps;
  ix->nyq_first = (int)h.nyq_first;
  ix->leaf_tiles = (int)h.leaf_tiles;
  ix->T = h.T;
  ix->L = h.L;
  ix->precision = (int)h.precision;
  ix->keybits = (int)h.keybits;
  ix->delta_d = h.delta_d;
  ix->delta_q = h.delta_q;
  ix->vmax = h.vmax;
  ix->outer = (float)h.outer;
  const Sizes z = sizes_of(ix);
  Staging sg;
  int64_t* acct = &ix->device_bytes;
  int rc = 0;
  rc = rc ? rc : read_array(f, sg, &ix->sel, z.nsel_i, false, acct);
  rc = rc ? rc : read_array(f, sg, &ix->sel_k, z.nsel_i, false, acct);
  rc = rc ? rc : read_array(f, sg, &ix->sel_part, z.nsel_i, false, acct);
  rc = rc ? rc : read_array(f, sg, &ix->var, z.nsel_d, false, acct);
  rc = rc ? rc : read_array(f, sg, &ix->basis, z.basis, false, acct);
  rc = rc ? rc : read_array(f, sg, &ix->beta, z.beta, false, acct);
  rc = rc ? rc : read_array(f, sg, &ix->edge, z.tab, false, acct);
  rc = rc ? rc : read_array(f, sg, &ix->ch, z.tab, false, acct);
  rc = rc ? rc : read_array(f, sg, &ix->ch16, z.tab / 2, false, acct);
  rc = rc ? rc : read_array(f, sg, &ix->words, z.words, false, acct);
  rc = rc ? rc : read_array(f, sg, &ix->Z, z.Z, false, acct);
  rc = rc ? rc : read_array(f, sg, &ix->perm, z.N4, false, acct);
  rc = rc ? rc : read_array(f, sg, &ix->keys, z.N8, false, acct);
  rc = rc ? rc : read_array(f, sg, &ix->keyorder, z.keyorder, false, acct);
  rc = rc ? rc : read_array(f, sg, &ix->tenv, z.tenv, false, acct);
  rc = rc ? rc : read_array(f, sg, &ix->lenv, z.lenv, false, acct);
  rc = rc ? rc : read_array(f, sg, &ix->xn, z.N4, false, acct);
  rc = rc ? rc : read_array(f, sg, &ix->Z8, z.Z8, true, acct);
  rc = rc ? rc : read_array(f, sg, &ix->s8, z.N4, true, acct);
  rc = rc ? rc : read_array(f, sg, &ix->e8, z.N4, true, acct);
  rc = rc ? rc : read_array(f, sg, &ix->VC, z.VC, true, acct);
  rc = rc ? rc : read_array(f, sg, &ix->vsr, z.vsr, true, acct);
  rc = rc ? rc : read_array(f, sg, &ix->vw, z.vw, true, acct);
  rc = rc ? rc : read_array(f, sg, &ix->Zh, z.Zh, true, acct);
  if (rc) return rc;
  if (!ix->Z8 != !ix->VC) return fail(SOFA_ERR_INVALID_ARG, "index file holds only part of the precision copies");
  if (int rc2 = make_tc_codes(ix, st)) return rc2;  // derived from the value codes, not stored
  SOFA_CUDA(cudaStreamSynchronize(st));
  if (h.has_mlp)
    if (int rc2 = mlp_load(ix, f, st)) return rc2;
  return 0;
}

}  // namespace
}  // namespace sofa

using namespace sofa;

extern "C" int sofa_save(sofa_handle h, const char* path) {
  if (!h || !path) return fail(SOFA_ERR_INVALID_ARG, "null argument");
  SOFA_CUDA(cudaDeviceSynchronize());
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(SOFA_ERR_INVALID_ARG, std::string("cannot open ") + path + " for writing");
  int rc = save_index(h, f);
  if (std::fclose(f) != 0 && !rc) rc = fail(SOFA_ERR_INVALID_ARG, "write failed");
  if (rc) std::remove(path);
  return rc;
}

extern "C" sofa_handle sofa_load(const char* path, sofa_stream stream) {
  if (!path) {
    set_error("path is NULL");
    return nullptr;
  }
  FILE* f = std::fopen(path, "rb");
  if (!f) {
    set_error(std::string("cannot open ") + path);
    return nullptr;
  }
  sofa_index* ix = new (std::nothrow) sofa_index();
  if (!ix) {
    std::fclose(f);
    set_error("host allocation failed");
    return nullptr;
  }
  cudaGetDevice(&ix->device);
  const int rc = load_index(ix, f, (cudaStream_t)stream);
  std::fclose(f);
  if (rc) {
    destroy_index(ix);
    return nullptr;
  }
  return ix;
}
