// Checkpoint / resume of a solve, one frequency at a time.  Algorithm 1 writes each task's output as
// it finishes, and the Evaluation section restarts long jobs from what is on disk; here each finished
// frequency's G block (all orbital rows and columns) is appended to a file, and a call with the same
// file and the same request restores the finished frequencies and solves the others.
//
// File (host byte order): "GFCCCKP1", int32 n_omega, n_orb, sectors, precision, rhf; double eta, tol;
// double omegas[n_omega]; int32 orbitals[n_orb]; then records {int32 w, int32 code, double G[2 n_orb^2]}.
// A record that was cut short (a job killed while writing) is dropped on resume.
#include <unistd.h>

#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ctx.cuh"

namespace gfcc {

namespace {

constexpr char MAGIC[8] = {'G', 'F', 'C', 'C', 'C', 'K', 'P', '1'};

struct Header {
  int n_omega = 0, n_orb = 0, sectors = 0, precision = 0, rhf = 0;
  double eta = 0.0, tol = 0.0;
  std::vector<double> omegas;
  std::vector<int> orbitals;
};

bool write_header(FILE *f, const Header &h) {
  const int ints[5] = {h.n_omega, h.n_orb, h.sectors, h.precision, h.rhf};
  const double dbl[2] = {h.eta, h.tol};
  return fwrite(MAGIC, 1, 8, f) == 8 && fwrite(ints, sizeof(int), 5, f) == 5 && fwrite(dbl, sizeof(double), 2, f) == 2 &&
         fwrite(h.omegas.data(), sizeof(double), h.omegas.size(), f) == h.omegas.size() &&
         fwrite(h.orbitals.data(), sizeof(int), h.orbitals.size(), f) == h.orbitals.size();
}

// 1: header read; 0: not a checkpoint of this format (or cut short)
int read_header(FILE *f, Header &h) {
  char m[8];
  int ints[5];
  double dbl[2];
  if (fread(m, 1, 8, f) != 8 || memcmp(m, MAGIC, 8) != 0) return 0;
  if (fread(ints, sizeof(int), 5, f) != 5 || fread(dbl, sizeof(double), 2, f) != 2) return 0;
  if (ints[0] < 0 || ints[1] < 0 || ints[0] > (1 << 24) || ints[1] > (1 << 20)) return 0;
  h.n_omega = ints[0];
  h.n_orb = ints[1];
  h.sectors = ints[2];
  h.precision = ints[3];
  h.rhf = ints[4];
  h.eta = dbl[0];
  h.tol = dbl[1];
  h.omegas.resize(h.n_omega);
  h.orbitals.resize(h.n_orb);
  if (fread(h.omegas.data(), sizeof(double), h.n_omega, f) != (size_t)h.n_omega) return 0;
  if (fread(h.orbitals.data(), sizeof(int), h.n_orb, f) != (size_t)h.n_orb) return 0;
  return 1;
}

bool same_request(const Header &a, const Header &b) {
  return a.n_omega == b.n_omega && a.n_orb == b.n_orb && a.sectors == b.sectors && a.precision == b.precision &&
         a.rhf == b.rhf && a.eta == b.eta && a.tol == b.tol && a.omegas == b.omegas && a.orbitals == b.orbitals;
}

int durable(FILE *f) {
  if (fflush(f) != 0) return -1;
  return fsync(fileno(f));
}

}  // namespace

int solve_checkpoint(gfcc_ctx *c, int n_omega, const double *omegas, double eta, int n_orb, const int *orbitals,
                     double tol, const char *path, int *n_resumed, double *G) {
  if (n_resumed) *n_resumed = 0;
  if (c == nullptr || path == nullptr || G == nullptr || omegas == nullptr || orbitals == nullptr || n_omega < 0 ||
      n_orb < 0) {
    set_error("gfcc_solve_checkpoint: need a context, a path, omegas, orbitals and G");
    return GFCC_ERR_ARG;
  }
  if (!(eta > 0.0) || !(tol > 0.0)) {
    set_error("gfcc_solve_checkpoint: need eta > 0 and tol > 0");
    return GFCC_ERR_ARG;
  }
  for (int a = 0; a < n_orb; a++)
    if (orbitals[a] < 0 || orbitals[a] >= c->n) {
      set_error("gfcc_solve_checkpoint: orbital index %d out of range [0, %d)", orbitals[a], c->n);
      return GFCC_ERR_ARG;
    }
  Header want;
  want.n_omega = n_omega;
  want.n_orb = n_orb;
  want.sectors = c->sectors;
  want.precision = c->precision;
  want.rhf = c->rhf;
  want.eta = eta;
  want.tol = tol;
  want.omegas.assign(omegas, omegas + n_omega);
  want.orbitals.assign(orbitals, orbitals + n_orb);
  const size_t blk = 2 * (size_t)n_orb * n_orb;   // doubles of one frequency's G block
  std::vector<char> done(n_omega, 0);
  std::vector<int> codes(n_omega, GFCC_OK);
  int resumed = 0;
  // ---- restore the finished frequencies of an earlier run of the same request
  if (FILE *f = fopen(path, "rb")) {
    Header have;
    const int ok = read_header(f, have);
    if (!ok || !same_request(have, want)) {
      fclose(f);
      set_error("gfcc_solve_checkpoint: %s holds %s; remove it or use another path", path,
                ok ? "the checkpoint of a different request (frequencies, orbitals, eta, tol or context)"
                   : "no checkpoint of this format");
      return GFCC_ERR_ARG;
    }
    std::vector<double> row(blk);
    for (;;) {
      int rec[2];
      if (fread(rec, sizeof(int), 2, f) != 2) break;
      if (fread(row.data(), sizeof(double), blk, f) != blk) break;   // cut short: dropped
      const int w = rec[0];
      if (w < 0 || w >= n_omega || done[w]) continue;
      memcpy(G + (size_t)w * blk, row.data(), sizeof(double) * blk);
      done[w] = 1;
      codes[w] = rec[1];
      resumed++;
    }
    fclose(f);
  }
  // ---- rewrite the file with the header and the complete records only, then append as we go
  const std::string tmp = std::string(path) + ".tmp";
  FILE *f = fopen(tmp.c_str(), "wb");
  if (f == nullptr || !write_header(f, want)) {
    if (f) fclose(f);
    set_error("gfcc_solve_checkpoint: cannot write %s", tmp.c_str());
    return GFCC_ERR_ARG;
  }
  for (int w = 0; w < n_omega; w++) {
    if (!done[w]) continue;
    const int rec[2] = {w, codes[w]};
    if (fwrite(rec, sizeof(int), 2, f) != 2 || fwrite(G + (size_t)w * blk, sizeof(double), blk, f) != blk) {
      fclose(f);
      set_error("gfcc_solve_checkpoint: cannot write %s", tmp.c_str());
      return GFCC_ERR_ARG;
    }
  }
  if (durable(f) != 0 || fclose(f) != 0 || rename(tmp.c_str(), path) != 0) {
    set_error("gfcc_solve_checkpoint: cannot replace %s", path);
    return GFCC_ERR_ARG;
  }
  if (n_resumed) *n_resumed = resumed;
  f = fopen(path, "ab");
  if (f == nullptr) {
    set_error("gfcc_solve_checkpoint: cannot append to %s", path);
    return GFCC_ERR_ARG;
  }
  // ---- solve the others, one frequency per call, each block on disk before the next starts
  int status = GFCC_OK;
  for (int w = 0; w < n_omega; w++) {
    if (done[w]) {
      if (codes[w] == GFCC_WARN_NOT_CONVERGED) status = GFCC_WARN_NOT_CONVERGED;
      continue;
    }
    const int rc = solve_rows_host(c, 1, omegas + w, eta, n_orb, orbitals, tol, G + (size_t)w * blk);
    if (rc < 0) {
      fclose(f);
      return rc;
    }
    if (rc == GFCC_WARN_NOT_CONVERGED) status = rc;
    const int rec[2] = {w, rc};
    if (fwrite(rec, sizeof(int), 2, f) != 2 || fwrite(G + (size_t)w * blk, sizeof(double), blk, f) != blk ||
        durable(f) != 0) {
      fclose(f);
      set_error("gfcc_solve_checkpoint: cannot append to %s", path);
      return GFCC_ERR_ARG;
    }
  }
  fclose(f);
  return status;
}

}  // namespace gfcc

extern "C" int gfcc_solve_checkpoint(gfcc_ctx *ctx, int n_omega, const double *omegas, double eta, int n_orb,
                                     const int *orbitals, double tol, const char *path, int *n_resumed, double *G) {
  return gfcc::solve_checkpoint(ctx, n_omega, omegas, eta, n_orb, orbitals, tol, path, n_resumed, G);
}
