/* Mesh multiplication with interface elements on the device (Sec. 2.4,
 * Eq. mmu, Algorithm 3).
 *
 * A coarse hex8 mesh with zero-thickness interface elements is divided
 * ndivi times on the GPU, so that a fine mesh never has to be generated,
 * stored or uploaded by the host.  One level:
 *   - every hex8 is divided into 8 children by new nodes at its edge
 *     midpoints, face centres and centre (the isoparametric map at the
 *     midpoints of the reference cube: means of 2, 4 and 8 corners);
 *   - every interface element is divided into 4 by planes parallel to its
 *     normal: its lower and upper faces are divided as the hex faces they
 *     coincide with, its zero-length edges are not divided;
 *   - counts (Eq. mmu, n_e^0 the total element count):
 *     n_e = 8 n_e^0 - 4 n_ELINT^0,
 *     n_n = n_n^0 + (hex edges) + (hex faces) + (hexes);
 *   - numbering: the old nodes keep their ids, then one node per divided
 *     edge in the order in which the edges first appear over (hex, local
 *     edge), then one per face likewise, then one per hex centre in hex
 *     order; hex child (ci, cj, ck) of hex e is 8e + ci + 2cj + 4ck (ci along
 *     the hex's 0-1 edge, cj along 0-3, ck along 0-4) with the parent's ply;
 *     interface child (ci, cj) of interface c is 4c + ci + 2cj;
 *   - coordinates in FP64: 0.5 (Xa + Xb), 0.25 (((X0 + X1) + X2) + X3) and
 *     0.125 (X0 + ... + X7) summed left to right, corners in the local order
 *     of the hex where the edge or face first appears (results do not depend
 *     on the launch configuration: every run gives the same mesh);
 *   - a new node holds the constraint bits all its parent corners hold
 *     (bitwise AND) and is a contact-surface node when all its parent
 *     corners are; the surface list keeps the old entries in order, then the
 *     new surface nodes in ascending id.
 * Local edge and face order of a hex8 (node order as in pdn_mesh_desc):
 *   edges 01 12 23 30 45 56 67 74 04 15 26 37;
 *   faces 0123 4567 0154 1265 2376 3047. */
#ifndef PDN_MMU_H
#define PDN_MMU_H

#include <stdint.h>

#include "pdn.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pdn_refined pdn_refined;

typedef struct {
  int64_t n_nodes, n_hex, n_coh, n_surf; /* the divided mesh */
  int64_t n_edges, n_faces;              /* edges and faces divided by the last level */
  int32_t levels;                        /* ndivi */
  int32_t pad;
  double device_ms;                      /* device time of all levels (CUDA events) */
} pdn_refined_info;

/* Divide the mesh `coarse` (as for pdn_init_mesh; its ply angles are kept
 * for pdn_init_refined) ndivi times (0..6) on the current device, on
 * `stream` (a cudaStream_t; NULL = the legacy default stream).  The divided
 * mesh stays in device memory owned by *out.  Errors: PDN_E_ARG (ids out of
 * range, an interface face that is not a face of some hex, a divided mesh
 * whose node or element ids do not fit in 32 bits), PDN_E_OOM, PDN_E_CUDA;
 * on failure *out is NULL and pdn_refined_last_error(NULL) says why. */
int pdn_mesh_multiply(pdn_refined **out, const pdn_mesh_desc *coarse, int32_t ndivi, void *stream);

/* Sizes and timing of the divided mesh. */
int pdn_refined_get_info(const pdn_refined *r, pdn_refined_info *info);

/* Copy the divided mesh to host buffers sized from pdn_refined_get_info:
 * X [3][n_nodes], hex [n_hex][8], coh [n_coh][8], ply_of_hex [n_hex],
 * fixed [n_nodes], surf [n_surf].  Any pointer may be NULL (not copied). */
int pdn_refined_get(const pdn_refined *r, double *X, int32_t *hex, int32_t *coh, int8_t *ply_of_hex,
                    uint8_t *fixed, int32_t *surf);

/* pdn_init_mesh on the divided mesh (ply angles of the coarse mesh).  The
 * solver's set-up (lumped mass, element lengths, stable steps, CSR) runs on
 * the host, so the divided mesh is read back once here. */
int pdn_init_refined(pdn_ctx **out, const pdn_refined *r, const pdn_material *mat, const pdn_options *opt);

/* Release the divided mesh.  NULL is ignored. */
void pdn_refined_destroy(pdn_refined *r);

/* Message of the last error of r, or of the last failed pdn_mesh_multiply
 * in this thread when r is NULL. */
const char *pdn_refined_last_error(const pdn_refined *r);

#ifdef __cplusplus
}
#endif

#endif /* PDN_MMU_H */
