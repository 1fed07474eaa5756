#include "rcb_internal.cuh"
namespace rcb {
int gravity(rcb_tree *, double *, double *) { return RCB_ERR_STATE; }
}
