"""Sub-models of a workload: selected cells with their external events, without connections."""
import numpy as np
def submodel(model, spec, cells):
    """Cells `cells` of a model as a model of their own, with their external events and
    without connections (for open-loop comparison of sampled cells)."""
    from .model import Model, SimSpec
    cells = np.asarray(cells, np.int64)
    off = model.cv_offset
    cv_old = np.concatenate([np.arange(off[c], off[c + 1]) for c in cells])
    new_of_old = np.full(model.n_cv, -1, np.int64)
    new_of_old[cv_old] = np.arange(cv_old.size)
    sizes = off[cells + 1] - off[cells]
    new_off = np.concatenate([[0], np.cumsum(sizes)])

    def sel(cv_arr, *vals):
        keep = new_of_old[cv_arr] >= 0
        return (new_of_old[cv_arr[keep]],) + tuple(v[keep] for v in vals) + (keep,)

    hh = sel(model.hh_cv, model.gnabar, model.gkbar, model.gl)
    pas = sel(model.pas_cv, model.g_pas, model.e_pas)
    syn = sel(model.syn_cv, model.syn_tau, model.syn_e)
    st = sel(model.stim_cv, model.stim_t_on, model.stim_dur, model.stim_amp)
    syn_new = np.full(model.n_syn, -1, np.int64)
    syn_new[np.nonzero(syn[-1])[0]] = np.arange(int(syn[-1].sum()))
    m = Model(cv_offset=new_off, parent=model.parent[cv_old], length_um=model.length_um[cv_old],
              radius_um=model.radius_um[cv_old], cm=model.cm[cv_old], Ra=model.Ra[cv_old],
              branch_of_cv=model.branch_of_cv[cv_old],
              hh_cv=hh[0], gnabar=hh[1], gkbar=hh[2], gl=hh[3],
              pas_cv=pas[0], g_pas=pas[1], e_pas=pas[2],
              syn_cv=syn[0], syn_tau=syn[1], syn_e=syn[2],
              stim_cv=st[0], stim_t_on=st[1], stim_dur=st[2], stim_amp=st[3],
              detector_cv=new_of_old[model.detector_cv[cells]], threshold=model.threshold)
    ev_keep = syn_new[spec.ev_syn] >= 0 if spec.ev_syn.size else np.zeros(0, bool)
    s = SimSpec(dt=spec.dt, t_end=spec.t_end, epoch_steps=spec.epoch_steps,
                ev_syn=syn_new[spec.ev_syn[ev_keep]], ev_t=spec.ev_t[ev_keep], ev_w=spec.ev_w[ev_keep],
                name=spec.name + "-sub")
    return m, s, cv_old



def cell_sample(model, spec, n_cells):
    """The whole workload when n_cells <= 0 or >= its size, else its first n_cells cells
    (open loop, with their external events). Returns (model, spec, cells used)."""
    if n_cells <= 0 or n_cells >= model.n_cells:
        return model, spec, model.n_cells
    m, s, _ = submodel(model, spec, np.arange(n_cells))
    return m, s, n_cells
