"""Independent event-by-event tracer for a handful of superparticles.

Test infrastructure: a second, deliberately naive implementation of the
superparticle step (Sec. III of the paper) in pure Python with numpy float32
scalars and its own Philox4x32-10 (Salmon et al., SC'11).  It shares no code
with the C oracle; the tests require the two to produce bit-identical records
for a few particles over a few tens of steps (brute force on tiny inputs).

Only initial particles are traced (no pulse), which is enough to exercise
flights, vacuum reflection, interface transmission, scattering, energy
splitting, secondaries, removal, moments, flux and compaction.
"""
import math

import numpy as np

F = np.float32
MASK = 0xFFFFFFFF


def philox(c, k):
    c = list(c)
    k = list(k)
    for r in range(10):
        if r:
            k = [(k[0] + 0x9E3779B9) & MASK, (k[1] + 0xBB67AE85) & MASK]
        a = 0xD2511F53 * c[0]
        b = 0xCD9E8D57 * c[2]
        c = [((b >> 32) ^ c[1] ^ k[0]) & MASK, b & MASK,
             ((a >> 32) ^ c[3] ^ k[1]) & MASK, a & MASK]
    return c


def threshold(p):
    if not p > 0:
        return 0
    if p >= 1:
        return MASK
    return min(int(math.floor(p * 2.0 ** 32)), MASK)


def direction(word):
    return F((2 * (word >> 9) + 1) - (1 << 23)) * F(2.0 ** -23)


class Tracer:
    def __init__(self, wl, stack=0):
        st = wl.stacks[stack]
        self.wl, self.st, self.sidx = wl, st, stack
        self.key = [wl.seed & MASK, (wl.seed >> 32) & MASK]
        edges = [0]
        for c in st.layer_cells:
            edges.append(edges[-1] + c)
        self.edges = [F(e) * F(wl.dz) for e in edges]
        self.ncell = edges[-1]
        self.mat = list(st.layer_mat)
        ne = wl.n_e
        self.P, self.Q = {}, {}
        for m in range(st.v.shape[0]):
            for s in range(2):
                for k in range(1, ne + 1):
                    ti, te = float(st.tau_in[m, s, k - 1]), float(st.tau_el[m])
                    rin = 0.0 if math.isinf(ti) else 1.0 / ti
                    rel = 0.0 if math.isinf(te) else 1.0 / te
                    rate = rel + rin
                    self.P[m, s, k] = threshold(-math.expm1(-float(wl.dt) * rate))
                    self.Q[m, s, k] = threshold(rin / rate if rate > 0 else 0.0)
        self.T = {}
        for i in range(len(st.layer_cells) - 1):
            for d in range(2):
                for s in range(2):
                    for k in range(1, ne + 1):
                        self.T[i, d, s, k] = threshold(float(st.T[i, d, s, k - 1]))
        self.P0 = [threshold((1.0 + float(p)) / 2.0) for p in st.p0]
        self.parts = []
        self.next_id = 0
        self.step_no = 0
        self.counts = dict(absorbed=0, spawned=0, dropped=0, bath=0, iface=0, trans=0)
        self.flux = {}
        self.dens = {}
        self.gens = {}

    # ---- state helpers: a particle is a dict ----
    def load(self, recs, next_id):
        for r in recs:
            w = int(r["packed"])
            self.parts.append(dict(z=F(r["z"]), mu=F(r["mu"]),
                                   id=int(r["id"]) | ((w >> 21) << 32), k=w & 255,
                                   s=(w >> 8) & 1, l=(w >> 9) & 15, g=(w >> 13) & 255))
        self.next_id = next_id

    def rand(self, key, sub):
        # key: the carrier's slot (event, secondary and boundary words)
        ctr = [key & MASK, ((key >> 32) | (self.sidx << 16)) & MASK, self.step_no, sub]
        return philox(ctr, self.key)

    def cell(self, z):
        c = int(np.floor(F(z) / F(self.wl.dz)))
        return min(max(c, 0), self.ncell - 1)

    def fly(self, p, tau, key, sub0):
        tau = F(tau)
        hit = 0
        while True:
            lay = p["l"]
            w = self.st.v[self.mat[lay], p["s"], p["k"] - 1] * p["mu"]
            z1 = p["z"] + w * tau
            lo, hi = self.edges[lay], self.edges[lay + 1]
            if p["mu"] > 0 and z1 > hi:
                zb, up = hi, True
            elif p["mu"] < 0 and z1 < lo:
                zb, up = lo, False
            else:
                p["z"] = F(z1)
                return
            if hit == 8:
                p["z"] = zb
                return
            tau = F(tau - (zb - p["z"]) / w)
            if not tau > 0:
                tau = F(0.0)
            p["z"] = zb
            last = len(self.mat) - 1
            if (up and lay == last) or (not up and lay == 0):
                p["mu"] = -p["mu"]
            else:
                self.counts["iface"] += 1
                iface, d = (lay, 0) if up else (lay - 1, 1)
                ok = True
                if not (self.wl.flags & 4):
                    ok = self.rand(key, sub0 + hit)[0] < self.T[iface, d, p["s"], p["k"]]
                if ok:
                    p["l"] = lay + 1 if up else lay - 1
                    self.counts["trans"] += 1
                else:
                    p["mu"] = -p["mu"]
            hit += 1

    def add_flux(self, s, a, b):
        for f in range(min(a, b) + 1, max(a, b) + 1):
            key = (self.step_no // self.wl.moment_every, s, f)
            self.flux[key] = self.flux.get(key, 0) + (1 if b > a else -1)

    def step(self):
        wl = self.wl
        half = F(wl.dt) * F(0.5)
        n0 = len(self.parts)
        for i in range(n0):
            p = self.parts[i]
            if p["k"] == 0:
                continue
            c0 = self.cell(p["z"])
            self.fly(p, half, i, 0x600)
            grp = philox([i >> 2, (self.sidx << 16) & MASK, self.step_no, 0x400], self.key)
            m = self.mat[p["l"]]
            k = p["k"]
            x = [grp[i & 3], 0, 0, 0]
            if x[0] < self.P[m, p["s"], k]:
                x = [x[0]] + self.rand(i, 0x500)[1:]
                inel = x[1] < self.Q[m, p["s"], k]
                if k == 1 and (inel or wl.flags & 8):
                    p["k"] = 0
                    self.counts["absorbed"] += 1
                    self.counts["bath"] += 1
                    self.add_flux(p["s"], c0, self.cell(p["z"]))
                    continue
                p["mu"] = direction(x[2])
                if inel:
                    kp = 1 + ((x[3] * (k - 1)) >> 32)
                    p["k"] = kp
                    if wl.flags & 2:
                        self.counts["bath"] += k - kp
                    else:
                        y = self.rand(i, 0x501)
                        q = dict(z=p["z"], mu=direction(y[1]), id=None, k=k - kp,
                                 s=0 if y[0] < self.P0[m] else 1, l=p["l"],
                                 g=min(p["g"] + 1, 255))
                        cs = self.cell(q["z"])
                        before = (self.counts["iface"], self.counts["trans"])
                        self.fly(q, half, i, 0x700)
                        if len(self.parts) < self.st.capacity:
                            q["id"] = self.next_id
                            self.next_id += 1
                            self.parts.append(q)
                            self.counts["spawned"] += 1
                            self.add_flux(q["s"], cs, self.cell(q["z"]))
                        else:
                            self.counts["iface"], self.counts["trans"] = before
                            self.counts["dropped"] += 1
            self.fly(p, half, i, 0x610)
            self.add_flux(p["s"], c0, self.cell(p["z"]))
        if (self.step_no + 1) % wl.moment_every == 0:
            t = (self.step_no + 1) // wl.moment_every - 1
            for p in self.parts:
                if p["k"]:
                    key = (t, p["s"], p["k"], self.cell(p["z"]))
                    self.dens[key] = self.dens.get(key, 0) + 1
                    gk = (t, self.cell(p["z"]))
                    self.gens[gk] = self.gens.get(gk, 0) + p["g"]
        if (self.step_no + 1) % wl.compact_every == 0:
            self.parts = [p for p in self.parts if p["k"]]
        self.step_no += 1

    def records(self):
        out = np.zeros(len(self.parts), [("z", "<f4"), ("mu", "<f4"), ("id", "<u4"),
                                         ("packed", "<u4")])
        for i, p in enumerate(self.parts):
            out[i] = (p["z"], p["mu"], p["id"] & MASK,
                      p["k"] | (p["s"] << 8) | (p["l"] << 9) | (p["g"] << 13)
                      | ((p["id"] >> 32) << 21))
        return out
