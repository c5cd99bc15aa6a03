"""Host-side replay of a lowered plan (from ptn_plan_describe(detail=1)) in
NumPy, used by the CPU tests to check the planner and lowering logic against
the oracle without a GPU.  It follows the addressing rules of the step
descriptors literally (strides, slices, arenas, variant gather); it is test
code, not a product path."""
import numpy as np


def var_ids(desc, kraus_rows):
    cols = desc["var_cols"]
    out = np.zeros((kraus_rows.shape[0], max(len(cols), 1)), dtype=np.int64)
    for c, ent in enumerate(cols):
        for site, mul in ent:
            out[:, c] += kraus_rows[:, site].astype(np.int64) * mul
    return out


def _bits_offsets(strides, n):
    idx = np.arange(1 << n, dtype=np.int64)
    off = np.zeros(1 << n, dtype=np.int64)
    for p, s in enumerate(strides):
        off += ((idx >> p) & 1) * int(s)
    return off


def _runs(steps, schedule):
    """Groups of steps executed together: single steps, or with a schedule the
    fused runs (a small step followed by steps marked fuse_prev)."""
    i = 0
    while i < len(steps):
        k = i + 1
        if schedule is not None:
            while k < len(steps) and steps[k].get("fuse_prev", 0):
                k += 1
        yield steps[i:k]
        i = k


def _order(n_inst, schedule):
    return range(n_inst - 1, -1, -1) if schedule == "desc" else range(n_inst)


def cache_reps(desc, j, vids, chunk_traj):
    """Per cache slot of block j, the representative of every local trajectory:
    the first trajectory of the chunk with the same variants on the columns the
    planner lists for the slot (computed here from those lists directly)."""
    reps = []
    for cols in desc["blocks"][j]["cache_cols"]:
        first, rep = {}, []
        for tl, g in enumerate(chunk_traj):
            key = tuple(int(v) for v in vids[g, cols])
            rep.append(first.setdefault(key, tl))
        reps.append(rep)
    return reps


def run_block(desc, j, kraus_rows, net_traj, net_prefix, schedule=None, cache=False):
    """Marginals [n_net, 2^b] (complex64 arithmetic) of block j for the given
    networks (net_traj non-decreasing), one chunk holding all of them.

    schedule "asc" / "desc": every fused run of small steps is executed one
    instance at a time, each instance walking the whole run before the next
    starts (in ascending / descending instance order), the two extreme
    interleavings of a fused launch's CTAs; the result must not change.

    cache: intermediate caching as the planner marked it: a cached step is
    computed for its slot's representative trajectories only (the other
    instances of its output are filled with NaN) and every operand that records
    a slot reads the representative's instance."""
    blk = desc["blocks"][j]
    vt = np.array(desc["var_table"], dtype=np.float32).view(np.complex64)
    vids = var_ids(desc, kraus_rows)
    net_traj = np.asarray(net_traj)
    chunk_traj = []
    net_tl = np.zeros(len(net_traj), dtype=np.int64)
    for n, t in enumerate(net_traj):
        if not chunk_traj or chunk_traj[-1] != t:
            chunk_traj.append(int(t))
        net_tl[n] = len(chunk_traj) - 1
    n_traj, n_net = len(chunk_traj), len(net_traj)
    inst_of = {0: 1, 1: n_traj, 2: n_net}
    reps = cache_reps(desc, j, vids, chunk_traj) if cache else None
    arenas = [np.zeros(max(blk["arena_const"], 1), np.complex64),
              np.zeros(max(blk["arena_traj"] * n_traj, 1), np.complex64),
              np.zeros(max(blk["arena_net"] * n_net, 1), np.complex64)]

    def operand(d, out_cls, inst):
        tl = net = 0
        if out_cls == 2:
            net, tl = inst, net_tl[inst]
        elif out_cls == 1:
            tl = inst
        if d["mode"] == 0:
            var = vids[chunk_traj[tl], d["leaf_col"]] if d["leaf_col"] >= 0 else 0
            arr, base = vt, d["leaf_base"] + var * d["inst_size"]
        else:
            oi = 0 if d["cls"] == 0 else (tl if d["cls"] == 1 else net)
            if reps is not None and d["cls"] == 1 and d.get("cache", 0):
                oi = reps[d["cache"] - 1][tl]
            arr = arenas[d["arena"]]
            base = d["arena_off"] * inst_of[d["arena"]] + oi * d["inst_size"]
        for q, st in d["slices"]:
            base += ((int(net_prefix[net]) >> q) & 1) * st
        v = arr[base:base + d["inst_size"]]
        return np.conj(v) if d["conj"] else v

    def product(src, out_cls, inst):
        """The outer product of a virt step's factors, read now (as the
        consumer's operand pack forms it)."""
        oa = _bits_offsets(src["out_stride"][0], src["n_out"])
        ob = _bits_offsets(src["out_stride"][1], src["n_out"])
        return operand(src["ops"][0], out_cls, inst)[oa] * operand(src["ops"][1], out_cls, inst)[ob]

    def one(st, inst):
        oa = _bits_offsets(st["out_stride"][0], st["n_out"])
        ob = _bits_offsets(st["out_stride"][1], st["n_out"])
        ka = _bits_offsets(st["sum_stride"][0], st["n_sum"])
        kb = _bits_offsets(st["sum_stride"][1], st["n_sum"])
        size = 1 << st["n_out"]
        obase = st["out_off"] * inst_of[st["out_arena"]]
        ops = [operand(st["ops"][x], st["out_cls"], inst) for x in range(2)]
        if st.get("prod"):
            x = st["prod"] - 1
            ops[x] = product(blk["steps"][st["prod_src"]], st["out_cls"], inst)
            if st["ops"][x]["conj"]:
                ops[x] = np.conj(ops[x])
        A, B = ops
        val = (A[oa[:, None] + ka[None, :]] * B[ob[:, None] + kb[None, :]]).sum(axis=1)
        arenas[st["out_arena"]][obase + inst * size: obase + (inst + 1) * size] = val

    def skip(st):
        """A virt step is not executed: its output is poisoned with NaN."""
        size = 1 << st["n_out"]
        obase = st["out_off"] * inst_of[st["out_arena"]]
        arenas[st["out_arena"]][obase: obase + inst_of[st["out_cls"]] * size] = np.nan

    for run in _runs(blk["steps"], schedule):
        if len(run) == 1 and run[0].get("virt"):
            skip(run[0])
            continue
        if len(run) == 1:
            st = run[0]
            k = st.get("cache", 0) if reps is not None else 0
            for inst in range(inst_of[st["out_cls"]]):
                if k and reps[k - 1][inst] != inst:
                    size = 1 << st["n_out"]
                    obase = st["out_off"] * inst_of[st["out_arena"]] + inst * size
                    arenas[st["out_arena"]][obase:obase + size] = np.nan
                else:
                    one(st, inst)
            continue
        for inst in _order(inst_of[run[0]["out_cls"]], schedule):
            for st in run:
                one(st, inst)
    root = blk["root"]
    xo = _bits_offsets(root["x_stride"], blk["b"])
    marg = np.zeros((n_net, 1 << blk["b"]), dtype=np.float64)
    for n in range(n_net):
        R = operand(root["op"], 2, n)
        marg[n] = R[xo].real
    return marg


def run_expval(desc, kraus_rows, w, var_table=None, schedule=None):
    """Replay of the expectation-value plan (ptn_plan_describe(detail=2)):
    forward steps, root adjoint w(x) conj(psi(x)), reversed steps.  Returns
    (psi [n_traj, 2^n] in basis order, F [n_traj], {leaf: adjoint [n_traj, size]}).
    schedule: as in run_block."""
    ev = desc["expval"]
    n = desc["n_qubits"]
    vt = np.array(desc["var_table"] if var_table is None else var_table, dtype=np.float32).view(np.complex64)
    vids = var_ids(desc, kraus_rows)
    nt = kraus_rows.shape[0]
    inst_of = {0: 1, 1: nt, 2: 0, 3: nt, 4: nt}
    arenas = [np.zeros(max(ev["arena"][a] * max(inst_of[a], 1), 1), np.complex64) for a in range(5)]

    def operand(d, t):
        if d["mode"] == 0:
            var = vids[t, d["leaf_col"]] if d["leaf_col"] >= 0 else 0
            arr, base = vt, d["leaf_base"] + var * d["inst_size"]
        else:
            oi = 0 if d["cls"] == 0 else t
            arr, base = arenas[d["arena"]], d["arena_off"] * inst_of[d["arena"]] + oi * d["inst_size"]
        v = arr[base:base + d["inst_size"]]
        return np.conj(v) if d["conj"] else v

    def one(st, inst):
        oa = _bits_offsets(st["out_stride"][0], st["n_out"])
        ob = _bits_offsets(st["out_stride"][1], st["n_out"])
        ka = _bits_offsets(st["sum_stride"][0], st["n_sum"])
        kb = _bits_offsets(st["sum_stride"][1], st["n_sum"])
        size = 1 << st["n_out"]
        obase = st["out_off"] * inst_of[st["out_arena"]]
        A = operand(st["ops"][0], inst)
        B = operand(st["ops"][1], inst)
        arenas[st["out_arena"]][obase + inst * size: obase + (inst + 1) * size] = \
            (A[oa[:, None] + ka[None, :]] * B[ob[:, None] + kb[None, :]]).sum(axis=1)

    def execute(steps):
        for run in _runs(steps, schedule):
            if len(run) == 1:
                for inst in range(inst_of[run[0]["out_cls"]]):
                    one(run[0], inst)
                continue
            for inst in _order(inst_of[run[0]["out_cls"]], schedule):
                for st in run:
                    one(st, inst)

    execute(ev["steps"])
    root = ev["root"]
    xo = _bits_offsets(root["x_stride"], n)
    psi = np.zeros((nt, 1 << n), np.complex64)
    size = root["op"]["inst_size"]
    for t in range(nt):
        R = operand(root["op"], t)
        psi[t] = R[xo]
        adj = arenas[3][ev["root_adj_off"] * nt + t * size: ev["root_adj_off"] * nt + (t + 1) * size]
        adj[xo] = (w * np.conj(psi[t])).astype(np.complex64)
    F = (np.abs(psi.astype(np.complex128)) ** 2 * w[None, :]).sum(axis=1)
    execute(ev["bwd"])
    grads = {}
    for p in ev["pleaves"]:
        base = p["lgrad_off"] * nt
        grads[p["leaf"]] = arenas[4][base: base + nt * p["size"]].reshape(nt, p["size"]).copy()
    return psi, F, grads
