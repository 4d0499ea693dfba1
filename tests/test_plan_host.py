"""The direction planner (paper_2607_03226_b300/csrc/plan.cpp) on the host:
mesh.cpp and plan.cpp compiled with the host C++ compiler and a small driver,
no GPU.  For every direction the driver replays the plan's level order
against a value ring: each position's inflow references must name, face by
face, the slot that the upstream neighbour across that face wrote in an
earlier level and that no cell has overwritten since (or an import for a wall
or lagged face), and every cell must appear exactly once.  This is what makes
the level-ordered sweep the triangular solve of Eq. (13).  It is checked for
untilted levels, for the default plan and for the forced tilt (release levels
along the mesh's long axis on every direction), and the default plan's tilt
must cut the ring on a FinFET mesh without exceeding the level cap."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2607_03226_b300", "csrc")
INCLUDE = os.path.join(ROOT, "include")

DRIVER = r"""
#include <cmath>
#include <cstdio>
#include <fstream>
#include <vector>
#include "nbte_internal.h"
namespace nbte {
void set_error(const std::string&) {}
bool test_timeouts() { return false; }
unsigned long long wait_limit_or(unsigned long long d) { return d; }
}
using namespace nbte;
template <typename T> std::vector<T> rd(std::ifstream& f, size_t n) {
  std::vector<T> v(n); f.read((char*)v.data(), n * sizeof(T)); return v;
}
int main(int argc, char** argv) {
  std::ifstream f(argv[1], std::ios::binary);
  int64_t hd[8]; f.read((char*)hd, sizeof(hd));
  const int dim = (int)hd[0], ctype = (int)hd[1];
  const int64_t nn = hd[2], nc = hd[3], nvc = hd[4], nbf = hd[5], nvf = hd[6], D = hd[7];
  auto xyz = rd<double>(f, nn * dim); auto cells = rd<int64_t>(f, nc * nvc); auto bf = rd<int64_t>(f, nbf * nvf);
  auto bt = rd<int32_t>(f, nbf); auto s = rd<double>(f, D * 3); auto w = rd<double>(f, D);
  int64_t nb; f.read((char*)&nb, 8); auto raw = rd<double>(f, nb * 4);
  std::vector<BC> bcs;
  for (int k = 0; k < nb; ++k) bcs.push_back({(int32_t)raw[4 * k], (int32_t)raw[4 * k + 1], raw[4 * k + 2], raw[4 * k + 3]});
  Mesh m;
  Status st = build_mesh(dim, nn, xyz.data(), ctype, nc, cells.data(), nbf, bf.data(), bt.data(), m);
  if (!st.good()) { std::printf("ERROR mesh %s\n", st.msg.c_str()); return 1; }
  Plan P;
  st = build_plan(m, (int)D, s.data(), w.data(), bcs, 300.0, P, 4);
  if (!st.good()) { std::printf("ERROR plan %s\n", st.msg.c_str()); return 1; }
  const int64_t N = m.n_cells;
  const int nfc = m.nfc, K = P.K;
  long long bad = 0;
  std::vector<int32_t> slot_cell(P.max_slots + 2), slot_level(P.max_slots + 2), seen(N);
  for (int i = 0; i < D; ++i) {
    std::fill(slot_cell.begin(), slot_cell.end(), -1);
    std::fill(slot_level.begin(), slot_level.end(), -1);
    std::fill(seen.begin(), seen.end(), 0);
    const int L = (int)(P.lvl_off[i + 1] - P.lvl_off[i] - 1);
    const int32_t* lp = P.level_ptr.data() + P.lvl_off[i];
    const size_t base = (size_t)i * N;
    for (int l = 0; l < L; ++l) {
      for (int32_t p = lp[l]; p < lp[l + 1]; ++p) {   // reads of level l
        const int32_t c = P.pos_cell[base + p];
        seen[c]++;
        int kk = 0;
        for (int k = 0; k < nfc; ++k) {
          const int64_t h = (int64_t)c * nfc + k;
          double a = 0, ar = 0;
          for (int d = 0; d < dim; ++d) { a += s[i * 3 + d] * m.An[h * dim + d]; ar += m.An[h * dim + d] * m.An[h * dim + d]; }
          if (!(a < -1e-12 * std::sqrt(ar))) continue;   // not an inflow face
          const int32_t ref = P.pos_ref[((size_t)i * K + kk) * N + p];
          ++kk;
          if (ref > 0) {
            if (m.nb[h] < 0 || slot_cell[ref] != (int32_t)m.nb[h] || !(slot_level[ref] < l)) ++bad;
          } else if (ref == 0) {
            ++bad;
          }
        }
      }
      for (int32_t p = lp[l]; p < lp[l + 1]; ++p) {   // then its writes
        const int32_t sl = P.pos_slot[base + p];
        if (sl > 0) { slot_cell[sl] = P.pos_cell[base + p]; slot_level[sl] = l; }
      }
    }
    for (int64_t c = 0; c < N; ++c) if (seen[c] != 1) ++bad;
    std::printf("DIR %d %d %d\n", i, L, P.n_slots[i]);
  }
  std::printf("SUMMARY %lld %d %d %lld\n", bad, P.max_levels, P.max_slots, (long long)P.lagged_faces);
  return 0;
}
"""


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("plan")
    (d / "driver.cpp").write_text(DRIVER)
    exe = d / "driver"
    subprocess.run([cxx, "-std=c++17", "-O2", "-I", CSRC, "-I", INCLUDE, str(d / "driver.cpp"),
                    os.path.join(CSRC, "mesh.cpp"), os.path.join(CSRC, "plan.cpp"), "-o", str(exe), "-lpthread"],
                   check=True)
    return exe, d


def _dump(p, path):
    m = p.mesh
    cells = np.ascontiguousarray(m.cells, np.int64)
    bf = np.ascontiguousarray(m.bfaces, np.int64)
    s = np.zeros((p.n_dirs, 3))
    s[:, :p.s.shape[1]] = p.s
    with open(path, "wb") as f:
        np.array([m.dim, m.cell_type, m.nodes.shape[0], cells.shape[0], cells.shape[1], bf.shape[0], bf.shape[1],
                  p.n_dirs], np.int64).tofile(f)
        np.ascontiguousarray(m.nodes[:, :m.dim], np.float64).tofile(f)
        cells.tofile(f)
        bf.tofile(f)
        np.ascontiguousarray(m.btags, np.int32).tofile(f)
        s.tofile(f)
        np.ascontiguousarray(p.w, np.float64).tofile(f)
        np.array([len(p.boundaries)], np.int64).tofile(f)
        np.array([[b.tag, b.type, b.T_wall, b.specularity] for b in p.boundaries], np.float64).tofile(f)


def _plan(driver, p, tilt):
    exe, d = driver
    path = d / f"{p.name}_{p.n_cells}.bin"
    if not path.exists():
        _dump(p, path)
    env = dict(os.environ)
    env.pop("NBTE_PLAN_TILT", None)
    if tilt is not None:
        env["NBTE_PLAN_TILT"] = tilt
    r = subprocess.run([str(exe), str(path)], capture_output=True, text=True, env=env, check=True)
    dirs = {}
    for line in r.stdout.splitlines():
        f = line.split()
        if f[0] == "DIR":
            dirs[int(f[1])] = (int(f[2]), int(f[3]))
        elif f[0] == "SUMMARY":
            summary = dict(bad=int(f[1]), max_levels=int(f[2]), max_slots=int(f[3]), lagged=int(f[4]))
    return summary, dirs


def _cases():
    from cases import CASES, tets_cyclic
    return [CASES["fin3d_tets"](), CASES["fin2d_mixed"](), CASES["cube_hex"](), tets_cyclic(),
            W.problems.finfet3d(h=8e-9, B=2, n_pol=4, n_az=8)]


@pytest.mark.parametrize("tilt", ["0", None, "force"])
def test_plan_replays_as_a_valid_sweep(driver, tilt):
    for p in _cases():
        summary, dirs = _plan(driver, p, tilt)
        assert summary["bad"] == 0, (p.name, p.n_cells, tilt, summary)
        assert len(dirs) == p.n_dirs


def test_tilted_fronts_cut_the_ring(driver):
    """On the 140k-tet FinFET (the 1.14M-tet workload's geometry at 4 nm
    cells) the default plan tilts the wide-front directions: fewer ring slots
    at most, and no direction longer than the longest untilted one."""
    p = W.problems.finfet3d(h=4e-9, B=2, n_pol=10, n_az=20)
    flat, dflat = _plan(driver, p, "0")
    tilt, dtilt = _plan(driver, p, None)
    assert flat["bad"] == 0 and tilt["bad"] == 0
    assert tilt["max_levels"] == flat["max_levels"]
    assert all(dtilt[i][1] <= dflat[i][1] for i in dflat)
    mean_flat = np.mean([v[1] for v in dflat.values()])
    mean_tilt = np.mean([v[1] for v in dtilt.values()])
    print(f"ring slots: max {flat['max_slots']} -> {tilt['max_slots']}, mean {mean_flat:.0f} -> {mean_tilt:.0f}")
    assert tilt["max_slots"] < 0.75 * flat["max_slots"]
    assert mean_tilt < 0.75 * mean_flat
