"""Structures from external tools (Sec. 2.3, application workflow): a relaxed or simulated
structure is read from a file, mapped onto the lattice by hea_map_structure and analysed by
hea_sro_counts / hea_sro_alpha to give the target SRO of a (larger) search.

File formats (text, no third-party reader):
  * LAMMPS data files, atom style "atomic" (orthogonal boxes): header counts, box bounds, an
    optional Masses section, and the Atoms section "id type x y z [ix iy iz]".  LAMMPS atom types
    1..T become species 0..T-1.
  * Plain XYZ: the atom count, a comment line, then one "label x y z" line per atom; integer labels
    are species indices, other labels (element symbols) are numbered in order of first appearance
    unless a `labels` list fixes the order.
Reading and writing are host-side file handling; every computation on the structure runs in
libhea's kernels.
"""
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from . import hea


@dataclass
class Structure:
    xyz: np.ndarray                 # [n][3] Cartesian positions
    species: np.ndarray             # [n] species indices (uint8)
    box_lo: np.ndarray              # [3]
    box_hi: np.ndarray              # [3]
    labels: List[str] = field(default_factory=list)   # species index -> label, when known

    @property
    def n(self) -> int:
        return int(self.species.shape[0])


def read_lammps_data(path: str) -> Structure:
    with open(path) as fh:
        lines = fh.read().splitlines()
    n_atoms = None
    lo = np.zeros(3)
    hi = np.zeros(3)
    i = 1   # the first line is a comment
    section = None
    atoms = []
    while i < len(lines):
        raw = lines[i].split("#")[0].strip()
        i += 1
        if not raw:
            continue
        words = raw.split()
        if section is None:
            if len(words) >= 2 and words[1] == "atoms":
                n_atoms = int(words[0])
                continue
            if len(words) >= 3 and words[1] == "atom" and words[2] == "types":
                continue
            if len(words) == 4 and words[2].endswith("lo") and words[3].endswith("hi"):
                axis = "xyz".index(words[2][0])
                lo[axis], hi[axis] = float(words[0]), float(words[1])
                continue
            if len(words) >= 3 and words[-3:] == ["xy", "xz", "yz"]:
                raise ValueError("triclinic boxes are not supported (the lattice is cubic)")
            if words[0] in ("Masses", "Atoms", "Velocities"):
                section = words[0]
                continue
            continue
        if words[0] in ("Masses", "Atoms", "Velocities", "Bonds", "Angles"):
            section = words[0]
            continue
        if section == "Atoms":
            if len(words) < 5:
                raise ValueError(f"{path}: Atoms line '{raw}' is not 'id type x y z' (atom style atomic)")
            atoms.append((int(words[0]), int(words[1]), float(words[2]), float(words[3]), float(words[4])))
    if n_atoms is None or len(atoms) != n_atoms:
        raise ValueError(f"{path}: header announces {n_atoms} atoms, Atoms section has {len(atoms)}")
    atoms.sort()
    arr = np.array([a[1:] for a in atoms], dtype=np.float64).reshape(-1, 4)
    types = arr[:, 0].astype(np.int64)
    if types.min() < 1 or types.max() > 255:
        raise ValueError(f"{path}: atom types must be 1..255")
    return Structure(arr[:, 1:4].copy(), (types - 1).astype(np.uint8), lo, hi)


def write_lammps_data(path: str, st: Structure, masses: Optional[List[float]] = None, comment: str = "hea structure"):
    n_types = int(st.species.max()) + 1 if st.n else 1
    with open(path, "w") as fh:
        fh.write(f"{comment}\n\n{st.n} atoms\n{n_types} atom types\n\n")
        for axis, name in enumerate("xyz"):
            fh.write(f"{st.box_lo[axis]:.10f} {st.box_hi[axis]:.10f} {name}lo {name}hi\n")
        if masses:
            fh.write("\nMasses\n\n")
            for t, m in enumerate(masses[:n_types]):
                fh.write(f"{t + 1} {m}\n")
        fh.write("\nAtoms # atomic\n\n")
        for i in range(st.n):
            x, y, z = st.xyz[i]
            fh.write(f"{i + 1} {int(st.species[i]) + 1} {x:.10f} {y:.10f} {z:.10f}\n")


def read_xyz(path: str, labels: Optional[List[str]] = None, box_lo=(0.0, 0.0, 0.0), box_hi=None) -> Structure:
    with open(path) as fh:
        lines = fh.read().splitlines()
    n = int(lines[0].split()[0])
    known = list(labels) if labels else []
    xyz = np.zeros((n, 3))
    sp = np.zeros(n, np.uint8)
    for i in range(n):
        w = lines[2 + i].split()
        lab = w[0]
        if lab.isdigit() and not labels:
            idx = int(lab)
        else:
            if lab not in known:
                if labels:
                    raise ValueError(f"{path}: label {lab} not in {labels}")
                known.append(lab)
            idx = known.index(lab)
        sp[i] = idx
        xyz[i] = [float(w[1]), float(w[2]), float(w[3])]
    lo = np.asarray(box_lo, np.float64)
    hi = np.asarray(box_hi, np.float64) if box_hi is not None else xyz.max(axis=0)
    return Structure(xyz, sp, lo, hi, known)


def write_xyz(path: str, st: Structure, comment: str = "hea structure"):
    with open(path, "w") as fh:
        fh.write(f"{st.n}\n{comment}\n")
        for i in range(st.n):
            lab = st.labels[st.species[i]] if st.labels else str(int(st.species[i]))
            x, y, z = st.xyz[i]
            fh.write(f"{lab} {x:.10f} {y:.10f} {z:.10f}\n")


def lattice_constant(st: Structure, lat: "hea.Lattice") -> float:
    """Cubic lattice constant implied by the box: box length / cells, equal on the three axes."""
    ext = np.asarray(st.box_hi) - np.asarray(st.box_lo)
    a = ext / np.asarray(lat.L, np.float64)
    if not np.allclose(a, a[0], rtol=1e-6):
        raise ValueError(f"box {ext} is not {lat.L} cubic cells of one lattice constant")
    return float(a[0])


def map_onto_lattice(st: Structure, lat: "hea.Lattice", S: int, a: Optional[float] = None, tol: float = 0.25,
                     stream=None):
    """Maps the structure onto the lattice on the GPU; returns (types device tensor, report[4] numpy).
    Raises ValueError unless every site gets exactly one atom of a valid species."""
    import torch
    if a is None:
        a = lattice_constant(st, lat)
    xyz = torch.as_tensor(np.ascontiguousarray(st.xyz, np.float64)).cuda()
    sp = torch.as_tensor(np.ascontiguousarray(st.species, np.uint8)).cuda()
    types = torch.empty(lat.N, dtype=torch.uint8, device="cuda")
    scratch = torch.empty(lat.N, dtype=torch.int32, device="cuda")
    report = torch.empty(4, dtype=torch.int64, device="cuda")
    hea.hea_map_structure(lat, st.n, xyz, sp, S, a, st.box_lo, tol, types, scratch, report, stream)
    rep = report.cpu().numpy()
    if st.n != lat.N or rep.any():
        raise ValueError(f"structure does not fill the lattice one atom per site: {st.n} atoms for {lat.N} sites, "
                         f"off-lattice {rep[0]}, taken twice {rep[1]}, empty {rep[2]}, bad species {rep[3]}")
    return types, rep


def target_from_structure(st: Structure, lat: "hea.Lattice", obj_like_n_per=None, S: Optional[int] = None,
                          a: Optional[float] = None, tol: float = 0.25, stream=None):
    """Target SRO alpha[M][S][S] of an external structure (map, full recount, Eq. sro on the GPU).
    Returns (alpha numpy, counts numpy, composition list)."""
    import torch
    if S is None:
        S = int(st.species.max()) + 1
    types, _ = map_onto_lattice(st, lat, S, a, tol, stream)
    n_per = np.bincount(st.species, minlength=S).astype(np.int64) if obj_like_n_per is None else obj_like_n_per
    M = lat.M
    counts = torch.empty((M, S, S), dtype=torch.int32, device="cuda")
    hea.hea_sro_counts(lat, 1, types, S, counts, stream)
    obj = hea.Objective(n_per, np.ones(M), np.zeros((M, S, S)))
    alpha = torch.empty((M, S, S), dtype=torch.float64, device="cuda")
    f2 = torch.empty(1, dtype=torch.float64, device="cuda")
    hea.hea_sro_alpha(lat, obj, counts, alpha, f2, stream)
    return alpha.cpu().numpy(), counts.cpu().numpy(), [int(x) for x in n_per]
