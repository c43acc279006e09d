// Batched ensembles of independent systems (placeholder until the persistent
// ensemble kernel lands: every entry point reports NB_ERR_STATE).
#include "nb_internal.cuh"

extern "C" {

nb_status nb_ensemble_init(nb_ctx *, int32_t, const int64_t *, const double *, const double *, const double *,
                           const double *)
{
    return NB_ERR_STATE;
}

nb_status nb_ensemble_run(nb_ctx *, double) { return NB_ERR_STATE; }

nb_status nb_ensemble_energy(nb_ctx *, double *) { return NB_ERR_STATE; }

nb_status nb_ensemble_get_state(nb_ctx *, nb_state_view *) { return NB_ERR_STATE; }

}  // extern "C"
